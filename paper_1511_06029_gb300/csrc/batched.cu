// Batched apply of many uneven QTT operators (different d, ranks and numbers
// of right-hand sides) in one persistent launch per memory wave, the waves
// captured in one CUDA graph.
//
// Work list.  For one wave of operators the items are all (operator o, core
// step k, right-hand side c, chunk of 32*TN position pairs), ordered step-
// major: every operator's step-0 chunks, then every operator's step-1
// chunks, and so on.  Each item is the Algorithm 2 contraction of one chunk
// (all output ranks).  CTAs take items from a global counter in that order;
// item (o, k, ...) first waits until all chunks of (o, k-1) are done.  Those
// were taken earlier by CTAs that are already running and never wait on a
// later item, so the waits always end; they are bounded anyway (a clock
// budget, after which the kernel raises the status word to QTT_ERR_TIMEOUT
// and every CTA leaves).
//
// Per item the CTA stages the input chunk (r_k ranks x 2 x 32*TN positions)
// in shared memory with cp.async (L2 copies: the intermediate was written by
// other CTAs of this launch); the next item is taken before the current one
// is computed and, when its dependency is already complete, its copies are
// issued at once so they overlap the current item's arithmetic (otherwise it
// is waited for after the current item is published -- never before, which
// keeps the no-deadlock argument above).  The core of the current (operator,
// step) sits in shared memory while consecutive items share it.  Each warp
// computes a block of TB output ranks for the 32*TN pairs (TN consecutive
// pairs per lane) with FP32 multiply-adds (TF32 mode rounds each staged
// operand to TF32; cores are packed TF32-rounded).  TB = 2 ceil(r_out/16), so
// the eight warps cover all output ranks in one pass.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "checked.cuh"
#include "qtt_internal.h"
#include "step_lp.h"

namespace qtt {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxRank = 48;  // core + 3 chunk stages fit one CTA
constexpr int kMaxD = 30;

struct BOp {
  int d;
  int64_t N, nrhs, ld;
  const float *x;
  float *y;
  float *buf0, *buf1;
  const float *cores;  // packed [a][j][rpad][i] per core
  int ranks[kMaxD + 1];
  int rpad[kMaxD + 1];
  int64_t coff[kMaxD + 1];
};

// One (operator, step) of a wave.  Its chunks (32*TN position pairs of one
// right-hand side) are grouped into slices of `slice` chunks; slices are the
// work items.  first = index of its first slice, ntiles = number of slices.
struct BSeg {
  int op, k, dep;
  int64_t first, ntiles;
  int64_t chunks_per_rhs, nchunks;
  int slice;
  int pc;  // pairs per chunk: 32*TN times as many groups as the stage holds
};

struct BWave {
  const BOp *ops;
  const BSeg *segs;
  int nseg;
  int64_t total;
  unsigned *done;
  unsigned long long *next;
  int *status;
  int tf32;
  long long wait_budget;  // clock cycles
  int max_k;              // 2 x max input rank of the wave (rows of a chunk)
  int core_floats;        // shared floats reserved for one core (16-aligned)
};

__device__ __forceinline__ float tf32_rne_b(float x) {
  unsigned u = __float_as_uint(x);
  if ((u & 0x7f800000u) != 0x7f800000u) {
    u += 0x0fffu + ((u >> 13) & 1u);
    u &= 0xffffe000u;
  }
  return __uint_as_float(u);
}

__device__ __forceinline__ unsigned smem_u32b(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async4(unsigned dst, const void *src, int n) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src), "r"(n));
}
__device__ __forceinline__ void cp_async16b(unsigned dst, const void *src, int n) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(n));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait_n() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}
constexpr int kMaxStagesB = 3;  // chunk buffers per CTA (ring depth, 2 or 3)

// One work item, decoded.
struct Item {
  long long idx;
  int seg;
};

// Lane `lane` owns the TN consecutive pairs TN lane .. TN lane + TN - 1 of
// the item (one vector shared load per (a, j)); the warp owns output ranks
// b0 .. b0 + TB - 1 (TB even), read two at a time as one 16-byte broadcast
// load ((b, i=0), (b, i=1), (b+1, i=0), (b+1, i=1)).
template <int TN>
__device__ __forceinline__ void load_v(const float *p, float (&v)[TN]) {
  if constexpr (TN == 4) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else {
    const float2 t = *reinterpret_cast<const float2 *>(p);
    v[0] = t.x; v[1] = t.y;
  }
}

template <int TB, int TN>
__device__ __forceinline__ void rank_block(const float *sm, const float *sG, int rin, int rpad,
                                           int b0, int rout, int lane, int npair_chunk,
                                           float *out, int64_t N, int64_t q0, int k,
                                           int64_t npairs, bool round_out) {

  // acc2[t][m] = (output i = 0, output i = 1) of rank b0 + t at pair m: the
  // two coefficients (b, 0), (b, 1) sit side by side in the core row, so
  // each multiply-add is one two-lane FP32 FMA (each lane rounded as fmaf)
  float2 acc2[TB][TN];
#pragma unroll
  for (int t = 0; t < TB; ++t)
#pragma unroll
    for (int m = 0; m < TN; ++m) acc2[t][m] = make_float2(0.0f, 0.0f);
#pragma unroll 4
  for (int kk = 0; kk < 2 * rin; ++kk) {
    float v[TN];
    load_v<TN>(sm + (size_t)kk * npair_chunk + TN * lane, v);
    float2 vv[TN];
#pragma unroll
    for (int m = 0; m < TN; ++m) vv[m] = make_float2(v[m], v[m]);
    const float4 *g4 = reinterpret_cast<const float4 *>(sG + (kk * rpad + b0) * 2);
#pragma unroll
    for (int t2 = 0; t2 < TB / 2; ++t2) {
      // ranks past the padded row contribute nothing (rpad is a multiple of 4)
      const float4 g = b0 + 2 * t2 < rpad ? g4[t2] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float2 gp[2] = {make_float2(g.x, g.y), make_float2(g.z, g.w)};
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int m = 0; m < TN; ++m)
          acc2[2 * t2 + h][m] = __ffma2_rn(gp[h], vv[m], acc2[2 * t2 + h][m]);
    }
  }
  float acc[TB][2][TN];
#pragma unroll
  for (int t = 0; t < TB; ++t)
#pragma unroll
    for (int m = 0; m < TN; ++m) {
      acc[t][0][m] = acc2[t][m].x;
      acc[t][1][m] = acc2[t][m].y;
    }
  if (round_out) {
#pragma unroll
    for (int t = 0; t < TB; ++t)
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int m = 0; m < TN; ++m) acc[t][i][m] = tf32_rne_b(acc[t][i][m]);
  }
  const int64_t bit = (int64_t)1 << k, low = bit - 1;
  const int64_t qb = q0 + TN * lane;
#pragma unroll
  for (int t = 0; t < TB; ++t) {
    const int b = b0 + t;
    if (b >= rout) break;
    float *ob = out + (int64_t)b * N;
    // TN consecutive pairs are TN consecutive positions once 2^k >= 4; the
    // vector store also needs an aligned row (the caller's y may have any ld)
    const int64_t pv = ((qb & ~low) << 1) | (qb & low);
    const bool vec = k >= 2 && qb < npairs &&
                     ((reinterpret_cast<uintptr_t>(ob + pv) |
                       reinterpret_cast<uintptr_t>(ob + pv + bit)) &
                      (sizeof(float) * TN - 1)) == 0;
    if (vec) {
      const int64_t p0 = pv;
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        float *o = ob + p0 + (i ? bit : 0);
        if constexpr (TN == 4)
          *reinterpret_cast<float4 *>(o) =
              make_float4(acc[t][i][0], acc[t][i][1], acc[t][i][2], acc[t][i][3]);
        else
          *reinterpret_cast<float2 *>(o) = make_float2(acc[t][i][0], acc[t][i][1]);
      }
    } else {
#pragma unroll
      for (int m = 0; m < TN; ++m) {
        const int64_t q = qb + m;
        if (q >= npairs) continue;
        const int64_t p0 = ((q & ~low) << 1) | (q & low);
        ob[p0] = acc[t][0][m];
        ob[p0 + bit] = acc[t][1][m];
      }
    }
  }
}

// Segment holding `item` (all 32 lanes of warp 0): a 32-way search over the
// segments' first items (increasing), one parallel load per round, so ~3
// rounds for thousands of segments instead of a dozen dependent loads.
__device__ __forceinline__ int find_seg(const BWave &w, long long item) {
  const int lane = threadIdx.x & 31;
  int lo = 0, hi = w.nseg;  // segs[lo].first <= item < segs[hi].first
  while (hi - lo > 1) {
    const int step = (hi - lo + 31) / 32;
    const int idx = lo + lane * step;
    const bool pred = idx < hi && w.segs[idx].first <= item;
    const unsigned m = __ballot_sync(0xffffffffu, pred);  // a prefix of lanes; lane 0 set
    const int last = 31 - __clz(m);
    lo += last * step;
    hi = min(lo + step, hi);
  }
  return lo;
}

// Take the next slice (warp 0); -> s_item (idx >= w.total: none left).
__device__ __forceinline__ void fetch_slice(const BWave &w, Item *s_item) {
  if (threadIdx.x < 32) {
    long long idx = 0;
    if (threadIdx.x == 0) idx = (long long)atomicAdd(w.next, 1ull);
    idx = __shfl_sync(0xffffffffu, idx, 0);
    int seg = 0;
    if (idx < w.total) seg = find_seg(w, idx);
    if (threadIdx.x == 0) {
      s_item->idx = idx;
      s_item->seg = seg;
    }
  }
}

// Wait (thread 0, bounded) until the item's dependency is complete; returns
// through *s_abort whether the kernel must stop.
__device__ __forceinline__ void wait_item(const BWave &w, const Item &it, int *s_abort) {
  if (threadIdx.x == 0) {
    int abort = *(volatile int *)w.status != 0;
    const int dep = w.segs[it.seg].dep;
    if (!abort && dep >= 0) {
      const unsigned target = (unsigned)w.segs[dep].ntiles;
      const long long t0 = clock64();
      while (*(volatile unsigned *)(w.done + dep) < target) {
        if (*(volatile int *)w.status != 0) { abort = 1; break; }
        if (clock64() - t0 > w.wait_budget) {
          atomicCAS(w.status, 0, (int)QTT_ERR_TIMEOUT);
          abort = 1;
          break;
        }
        __nanosleep(64);
      }
      __threadfence();
    }
    *s_abort = abort;
  }
}

// Issue the asynchronous copies of chunk (c, q0) of step k into `buf`
// ([2a + j][pair], PC pairs per row): 16-byte copies when 4 consecutive
// pairs are 4 consecutive positions (k >= 2), 4-byte copies otherwise;
// pairs past the end are zero-filled.
__device__ __forceinline__ void stage_chunk(const BOp &op, int k, int64_t c, int64_t q0,
                                            int PC, float *buf) {
  const int rin = op.ranks[k];
  const int64_t N = op.N, npairs = N >> 1;
  const int64_t bit = (int64_t)1 << k, low = bit - 1;
  const float *in = k == 0 ? op.x + c * op.ld
                           : ((k - 1) & 1 ? op.buf1 : op.buf0) + c * (int64_t)rin * N;
  if (k >= 2) {
    const int PIECES = PC / 4;
    for (int e = threadIdx.x; e < 2 * rin * PIECES; e += kThreads) {
      const int kk = e / PIECES, pc = e % PIECES;
      const int64_t q = q0 + 4 * pc;
      const bool ok = q < npairs;
      const float *src = in + (int64_t)(kk >> 1) * N + (((q & ~low) << 1) | (q & low)) +
                         ((kk & 1) ? bit : 0);
      cp_async16b(smem_u32b(buf + kk * PC + 4 * pc), ok ? src : op.x, ok ? 16 : 0);
    }
  } else {
    for (int e = threadIdx.x; e < 2 * rin * PC; e += kThreads) {
      const int kk = e / PC, qq = e % PC;
      const int64_t q = q0 + qq;
      const bool ok = q < npairs;
      const float *src = in + (int64_t)(kk >> 1) * N + (((q & ~low) << 1) | (q & low)) +
                         ((kk & 1) ? bit : 0);
      cp_async4(smem_u32b(buf + kk * PC + qq), ok ? src : op.x, ok ? 4 : 0);
    }
  }
}

// The chunk's work units are (rank block of TB ranks, group of 32*TN pairs);
// warps take them round robin, so small output ranks (few rank blocks) still
// keep every warp busy on a wider chunk.
template <int TN, int TBMAX>
__device__ __forceinline__ void compute_chunk(const float *sb, const float *sG, int rin,
                                              int rpad, int rout, int warp, int lane, int PCe,
                                              float *out, int64_t N, int64_t q0, int k,
                                              int64_t npairs, bool round_out) {
  constexpr int GP = 32 * TN;  // pairs per group
  const int TB = rout <= 2 ? 2 : 2 * ((rout + 15) / 16);  // even, <= 6
  const int nb = (rout + TB - 1) / TB;
  const int units = nb * (PCe / GP);
  for (int u = warp; u < units; u += kThreads / 32) {
    const int b0 = (u % nb) * TB, g = u / nb;
    const float *sg = sb + g * GP;
    const int64_t qg = q0 + (int64_t)g * GP;
    switch (TB) {
      case 2: rank_block<2, TN>(sg, sG, rin, rpad, b0, rout, lane, PCe, out, N, qg, k, npairs, round_out); break;
      case 4: rank_block<4, TN>(sg, sG, rin, rpad, b0, rout, lane, PCe, out, N, qg, k, npairs, round_out); break;
      default: rank_block<6, TN>(sg, sG, rin, rpad, b0, rout, lane, PCe, out, N, qg, k, npairs, round_out); break;
    }
  }
}

template <int TN, int TBMAX, int NS>
__global__ void __launch_bounds__(kThreads) batch_kernel(BWave w) {
  extern __shared__ __align__(16) float sm[];
  constexpr int PC = 32 * TN;  // pairs per chunk
  __shared__ Item s_item;
  __shared__ int s_abort;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float *sG = sm;                              // core of the current segment
  float *sB = sm + w.core_floats;              // NS chunk buffers
  const size_t stage = (size_t)w.max_k * PC;
  int gseg = -1;                               // segment whose core is in sG
  for (;;) {
    fetch_slice(w, &s_item);
    __syncthreads();
    const Item it = s_item;
    if (it.idx >= w.total) break;
    wait_item(w, it, &s_abort);
    __syncthreads();
    if (s_abort) break;
    const BSeg sg = w.segs[QTT_CK(it.seg, w.nseg, 401)];
    const BOp &op = w.ops[sg.op];
    const int k = (int)QTT_CK(sg.k, op.d, 402);
    const int rin = op.ranks[k], rout = op.ranks[k + 1];
    const int rpad = op.rpad[k + 1];
    const int64_t N = op.N, npairs = N >> 1;
    if (gseg != it.seg) {
      const float *G = op.cores + op.coff[k];
      for (int e = tid; e < 2 * rin * 2 * rpad; e += kThreads) sG[e] = __ldg(G + e);
      gseg = it.seg;
    }
    const int64_t c_begin = QTT_CK((it.idx - sg.first) * sg.slice, sg.nchunks, 403);
    const int64_t c_end = c_begin + sg.slice < sg.nchunks ? c_begin + sg.slice : sg.nchunks;
    const bool round_in = w.tf32 && k == 0;          // x itself is not TF32-rounded
    const bool round_out = w.tf32 && k < op.d - 1;   // intermediates are stored rounded
    float *out_base = k == op.d - 1 ? op.y : (k & 1 ? op.buf1 : op.buf0);
    const int64_t out_stride = k == op.d - 1 ? op.ld : (int64_t)rout * N;
    // prologue: the first NS - 1 chunks of the slice
#pragma unroll
    for (int st = 0; st < NS - 1; ++st) {
      const int64_t t = c_begin + st;
      if (t < c_end) stage_chunk(op, k, t / sg.chunks_per_rhs,
                                 (t % sg.chunks_per_rhs) * sg.pc, sg.pc, sB + st * stage);
      cp_commit();
    }
    int cur = 0;
    for (int64_t t = c_begin; t < c_end; ++t) {
      {
        const int64_t tn = t + NS - 1;
        if (tn < c_end)
          stage_chunk(op, k, tn / sg.chunks_per_rhs, (tn % sg.chunks_per_rhs) * sg.pc, sg.pc,
                      sB + ((cur + NS - 1) % NS) * stage);
        cp_commit();
      }
      cp_wait_n<NS - 1>();
      __syncthreads();
      float *sb = sB + cur * stage;
      if (round_in) {
        for (int e = tid; e < 2 * rin * sg.pc; e += kThreads) sb[e] = tf32_rne_b(sb[e]);
        __syncthreads();
      }
      const int64_t c = t / sg.chunks_per_rhs, q0 = (t % sg.chunks_per_rhs) * sg.pc;
      compute_chunk<TN, TBMAX>(sb, sG, rin, rpad, rout, warp, lane, sg.pc,
                               out_base + c * out_stride, N, q0, k, npairs, round_out);
      __syncthreads();  // the stage is refilled next iteration
      cur = (cur + 1) % NS;
    }
    cp_wait_all();
    // publish the slice: the barrier above ordered every thread's stores
    // before thread 0's device-scope fence and counter update
    if (tid == 0) {
      __threadfence();
      atomicAdd(w.done + it.seg, 1u);
    }
  }
  cp_wait_all();
}

}  // namespace

// ------------------------------------------------------------------ host
struct WaveDev {
  std::vector<int> ops;
  BOp *d_ops = nullptr;
  BSeg *d_segs = nullptr;
  unsigned *d_done = nullptr;
  int nseg = 0;
  int64_t total = 0;
  int64_t first_dep = -1;  // index of the first item that waits on another
  int max_rin = 1;
};

}  // namespace qtt

namespace qtt {
// FP32 batches: operators with d at least this large go through the
// single-operator apply (staged FP32 steps), which keeps more of the FP32
// pipe busy than a shared wave once one operator fills the GPU
constexpr int kDirectMinD = 16;
}  // namespace qtt

struct qtt_batch {
  std::vector<const qtt_op *> ops;
  std::vector<int64_t> nrhs, ld;
  std::vector<const float *> x;
  std::vector<float *> y;
  qtt_dtype compute = QTT_F32;
  size_t budget = 0;
  int variant = 4;  // TN
  int slice = 8;    // chunks per work item
  int stages = 3;   // cp.async ring depth
  std::vector<qtt::WaveDev> waves;
  float *scratch = nullptr;
  size_t scratch_bytes = 0;
  unsigned long long *d_next = nullptr;  // one counter per wave
  int *d_status = nullptr;
  cudaEvent_t last_run = nullptr;  // recorded after each run (for destroy)
  // qtt_batch_selftest_timeout: start wave 0 at this item with this wait
  // budget (clock cycles), launching that wave alone (-1: normal runs)
  int64_t selftest_start = -1;
  long long selftest_budget = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  double flops = 0.0;
  int grid = 0;
  // operators applied with the single-operator apply after the waves, not in
  // a wave: TF32 ones whose apply runs tcgen05 step pairs, FP32 ones with
  // d >= kDirectMinD
  std::vector<int> direct_ops;
  // qtt_batch_run_host: events ordering the copies against the applies
  // (created on its first call; [0] start, [1] wave inputs in, [2] waves
  // done, [3] copies out done, then one pair per direct operator)
  std::vector<cudaEvent_t> host_events;
};

namespace qtt {
namespace {

size_t op_scratch_bytes(const qtt_op *A, int64_t nrhs) {
  if (A->d <= 1) return 0;
  return (size_t)2 * A->rmax_inner * ((size_t)1 << A->d) * (size_t)nrhs * sizeof(float);
}

// Device buffers of a batch come from the library's pool (persistent_alloc)
// and go back stream-ordered, after the batch's last run.
void release(qtt_batch *B, std::vector<void *> ptrs) {
  std::vector<cudaEvent_t> after;
  if (B->last_run) after.push_back(B->last_run);
  release_after(ptrs, after);
}

void free_waves(qtt_batch *B) {
  std::vector<void *> ptrs;
  for (auto &w : B->waves) {
    ptrs.push_back(w.d_ops);
    ptrs.push_back(w.d_segs);
    ptrs.push_back(w.d_done);
  }
  release(B, ptrs);
  B->waves.clear();
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  B->exec = nullptr;
  B->graph = nullptr;
}

qtt_status build_plan(qtt_batch *B, cudaStream_t st) {
  free_waves(B);
  const int TN = B->variant;
  const int PC = 32 * TN;
  // Waves hold operators of one rank class (largest rank <= 16, <= 24,
  // <= 32, <= 48), so that each wave's kernel is sized -- shared memory,
  // hence CTAs per SM -- for its own class; within a class, greedy waves in
  // input order under the memory budget.
  auto rank_class = [](const qtt_op *A) {
    int r = 1;
    for (int k = 0; k <= A->d; ++k) r = std::max(r, A->ranks[k]);
    return r <= 16 ? 0 : r <= 24 ? 1 : r <= 32 ? 2 : 3;
  };
  std::vector<int> order;
  B->direct_ops.clear();
  for (size_t i = 0; i < B->ops.size(); ++i) {
    const qtt_op *A = B->ops[i];
    if ((B->compute == QTT_TF32 && tf32_tc_pairs(A) > 0) ||
        (B->compute == QTT_F32 && A->d >= kDirectMinD))
      B->direct_ops.push_back((int)i);
    else
      order.push_back((int)i);
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return rank_class(B->ops[a]) < rank_class(B->ops[b]);
  });
  std::vector<std::vector<int>> groups;
  size_t cur = 0, maxw = 0;
  int cls = -1;
  for (int i : order) {
    const size_t need = op_scratch_bytes(B->ops[i], B->nrhs[i]);
    if (need > B->budget)
      return fail(QTT_ERR_OOM, "batch: one operator's scratch exceeds the memory budget");
    if (groups.empty() || cur + need > B->budget || rank_class(B->ops[i]) != cls) {
      groups.emplace_back();
      cur = 0;
      cls = rank_class(B->ops[i]);
    }
    groups.back().push_back(i);
    cur += need;
    maxw = std::max(maxw, cur);
  }
  if (B->scratch_bytes < maxw) {
    release(B, {B->scratch});
    B->scratch = nullptr;
    B->scratch_bytes = 0;
    if (maxw > scratch_available()) return fail(QTT_ERR_OOM, "batch: scratch does not fit");
    if (qtt_status as = persistent_alloc(reinterpret_cast<void **>(&B->scratch), maxw, st))
      return as;
    B->scratch_bytes = maxw;
  }
  release(B, {B->d_next});
  B->d_next = nullptr;
  if (qtt_status as = persistent_alloc(reinterpret_cast<void **>(&B->d_next),
                                       sizeof(unsigned long long) * std::max<size_t>(1, groups.size()), st))
    return as;
  for (auto &g : groups) {
    // the wave's kernel is sized for the largest rank of its own operators
    int max_rank_wave = 1;
    for (int i : g)
      for (int k = 0; k <= B->ops[i]->d; ++k) max_rank_wave = std::max(max_rank_wave, B->ops[i]->ranks[k]);
    const int max_k_wave = 2 * max_rank_wave;
    WaveDev wv;
    wv.ops = g;
    std::vector<BOp> hops;
    size_t off = 0;
    int maxd = 0;
    for (int i : g) {
      const qtt_op *A = B->ops[i];
      BOp o;
      std::memset(&o, 0, sizeof(o));
      o.d = A->d;
      o.N = (int64_t)1 << A->d;
      o.nrhs = B->nrhs[i];
      o.ld = B->ld[i];
      o.x = B->x[i];
      o.y = B->y[i];
      const size_t half = (size_t)A->rmax_inner * (size_t)o.N * (size_t)o.nrhs;
      o.buf0 = reinterpret_cast<float *>(reinterpret_cast<char *>(B->scratch) + off);
      o.buf1 = o.buf0 + half;
      off += op_scratch_bytes(A, o.nrhs);
      o.cores = B->compute == QTT_TF32 ? A->mtf32 : A->m32;
      for (int k = 0; k <= A->d; ++k) {
        o.ranks[k] = A->ranks[k];
        o.rpad[k] = A->rpad[k];
        o.coff[k] = A->offlp[k];
        wv.max_rin = std::max(wv.max_rin, A->ranks[k]);
      }
      hops.push_back(o);
      maxd = std::max(maxd, A->d);
    }
    // segments, step-major
    std::vector<BSeg> segs;
    std::vector<std::vector<int>> seg_of(g.size(), std::vector<int>(maxd, -1));
    int64_t first = 0;
    for (int k = 0; k < maxd; ++k)
      for (int li = 0; li < (int)g.size(); ++li) {
        const BOp &o = hops[li];
        if (k >= o.d) continue;
        BSeg s;
        s.op = li;
        s.k = k;
        s.dep = k > 0 ? seg_of[li][k - 1] : -1;
        // widen the chunk while the stage (max_k rows of PC pairs) holds it,
        // the pairs exist, and each warp would still get under 2 units
        {
          const int rows = 2 * o.ranks[k];
          int f = 1;
          while (rows * PC * (f * 2) <= max_k_wave * PC && (int64_t)PC * f * 2 <= (o.N >> 1) &&
                 f * 2 <= 64)
            f *= 2;
          s.pc = PC * f;
        }
        s.chunks_per_rhs = ((o.N >> 1) + s.pc - 1) / s.pc;
        s.nchunks = s.chunks_per_rhs * o.nrhs;
        s.slice = B->slice;
        s.ntiles = (s.nchunks + s.slice - 1) / s.slice;
        s.first = first;
        first += s.ntiles;
        seg_of[li][k] = (int)segs.size();
        segs.push_back(s);
      }
    wv.nseg = (int)segs.size();
    wv.total = first;
    for (const BSeg &sg : segs)
      if (sg.dep >= 0 && (wv.first_dep < 0 || sg.first < wv.first_dep)) wv.first_dep = sg.first;
    for (auto pr : {std::make_pair(reinterpret_cast<void **>(&wv.d_ops), sizeof(BOp) * hops.size()),
                    std::make_pair(reinterpret_cast<void **>(&wv.d_segs), sizeof(BSeg) * segs.size()),
                    std::make_pair(reinterpret_cast<void **>(&wv.d_done), sizeof(unsigned) * segs.size())})
      if (qtt_status as = persistent_alloc(pr.first, pr.second, st)) {
        release(B, {wv.d_ops, wv.d_segs, wv.d_done});
        return as;
      }
    QTT_CUDA_TRY(cudaMemcpyAsync(wv.d_ops, hops.data(), sizeof(BOp) * hops.size(),
                                 cudaMemcpyHostToDevice, st));
    QTT_CUDA_TRY(cudaMemcpyAsync(wv.d_segs, segs.data(), sizeof(BSeg) * segs.size(),
                                 cudaMemcpyHostToDevice, st));
    B->waves.push_back(wv);
  }
  QTT_CUDA_TRY(cudaStreamSynchronize(st));
  return QTT_OK;
}

template <int TN, int NS>
qtt_status launch_waves_t(qtt_batch *B, cudaStream_t st) {
  const int PC = 32 * TN;
  // raised once to the largest footprint (rank kMaxRank), shared by all threads
  static cudaError_t attr = cudaFuncSetAttribute(
      batch_kernel<TN, 6, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
      (int)(sizeof(float) * ((size_t)(2 * kMaxRank * 2 * kMaxRank) +
                             (size_t)NS * (2 * kMaxRank) * PC)));
  QTT_CUDA_TRY(attr);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int clk_khz = 2000000;
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
  // each wave sized for its own largest rank: shared memory and so the CTAs
  // resident per SM
  auto sizing = [&](const WaveDev &w, int *max_k, int *core_floats, size_t *smem, int *grid) {
    *max_k = 2 * w.max_rin;
    const int rpad_max = (w.max_rin + 3) / 4 * 4;
    *core_floats = (*max_k * 2 * rpad_max + 15) / 16 * 16;
    *smem = sizeof(float) * ((size_t)*core_floats + (size_t)NS * *max_k * PC);
    int per_sm = 0;
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, batch_kernel<TN, 6, NS>, kThreads, *smem);
    *grid = std::max(1, per_sm) * sms;
    return e;
  };
  B->grid = 0;
  for (const auto &w : B->waves) {
    int mk, cf, g;
    size_t sm;
    QTT_CUDA_TRY(sizing(w, &mk, &cf, &sm, &g));
    B->grid = std::max(B->grid, g);
  }
  const bool selftest = B->selftest_start >= 0;
  for (size_t wi = 0; wi < (selftest ? (size_t)1 : B->waves.size()); ++wi) {
    auto &w = B->waves[wi];
    QTT_CUDA_TRY(cudaMemsetAsync(w.d_done, 0, sizeof(unsigned) * w.nseg, st));
    if (selftest) {
      // the work list starts past every item without a dependency: the
      // items the others wait on are never taken
      const unsigned long long start = (unsigned long long)B->selftest_start;
      QTT_CUDA_TRY(cudaMemcpyAsync(B->d_next + wi, &start, sizeof(start), cudaMemcpyHostToDevice, st));
      QTT_CUDA_TRY(cudaStreamSynchronize(st));
    } else {
      QTT_CUDA_TRY(cudaMemsetAsync(B->d_next + wi, 0, sizeof(unsigned long long), st));
    }
    BWave bw;
    bw.ops = w.d_ops;
    bw.segs = w.d_segs;
    bw.nseg = w.nseg;
    bw.total = w.total;
    bw.done = w.d_done;
    bw.next = B->d_next + wi;
    bw.status = B->d_status;
    bw.tf32 = B->compute == QTT_TF32;
    bw.wait_budget = selftest ? B->selftest_budget : (long long)clk_khz * 1000LL * 4;  // ~4 s
    int max_k, core_floats, grid;
    size_t smem;
    QTT_CUDA_TRY(sizing(w, &max_k, &core_floats, &smem, &grid));
    bw.max_k = max_k;
    bw.core_floats = core_floats;
    batch_kernel<TN, 6, NS><<<grid, kThreads, smem, st>>>(bw);
    count_launches(1);
    QTT_CUDA_TRY(cudaGetLastError());
  }
  return QTT_OK;
}

qtt_status launch_waves(qtt_batch *B, cudaStream_t st) {
  const bool deep = B->stages == 3;
  switch (B->variant) {
    case 2: return deep ? launch_waves_t<2, 3>(B, st) : launch_waves_t<2, 2>(B, st);
    default: return deep ? launch_waves_t<4, 3>(B, st) : launch_waves_t<4, 2>(B, st);
  }
}

qtt_status capture(qtt_batch *B, cudaStream_t st) {
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  B->exec = nullptr;
  B->graph = nullptr;
  // Capture on a private stream so the caller's stream state is untouched.
  cudaStream_t cs;
  QTT_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    return cuda_fail(e, "batch: begin capture");
  }
  qtt_status s = launch_waves(B, cs);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(cs, &g);
  cudaStreamDestroy(cs);
  if (s != QTT_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) return cuda_fail(e, "batch: end capture");
  B->graph = g;
  e = cudaGraphInstantiate(&B->exec, g, 0);
  if (e != cudaSuccess) return cuda_fail(e, "batch: instantiate");
  (void)st;
  return QTT_OK;
}

}  // namespace
}  // namespace qtt

using namespace qtt;

extern "C" {

qtt_status qtt_batch_create(qtt_batch **out, int nops, const qtt_op *const *ops,
                            const int64_t *nrhs, const void *const *x, void *const *y,
                            const int64_t *ld, qtt_dtype compute, size_t mem_budget,
                            void *stream) {
  if (!out) return fail(QTT_ERR_INVALID_ARG, "qtt_batch_create: out is NULL");
  *out = nullptr;
  if (nops < 1 || !ops || !nrhs || !x || !y || !ld)
    return fail(QTT_ERR_INVALID_ARG, "qtt_batch_create: empty batch or NULL array");
  if (compute != QTT_F32 && compute != QTT_TF32)
    return fail(QTT_ERR_UNSUPPORTED, "qtt_batch_create: compute must be QTT_F32 or QTT_TF32");
  for (int i = 0; i < nops; ++i) {
    const qtt_op *A = ops[i];
    if (!A || !x[i] || !y[i]) return fail(QTT_ERR_INVALID_ARG, "qtt_batch_create: NULL entry");
    if (nrhs[i] < 1 || nrhs[i] > (int64_t)1 << 24)
      return fail(QTT_ERR_INVALID_ARG, "qtt_batch_create: nrhs out of range");
    if (ld[i] < ((int64_t)1 << A->d)) return fail(QTT_ERR_INVALID_ARG, "qtt_batch_create: ld < N");
    if (qtt_status ds = check_device(A, "qtt_batch_create")) return ds;
    if ((compute == QTT_F32 && !A->m32) || (compute == QTT_TF32 && !A->mtf32))
      return fail(QTT_ERR_INVALID_ARG, "qtt_batch_create: operator lacks the packed copy");
    for (int k = 0; k <= A->d; ++k)
      if (A->ranks[k] > kMaxRank)
        return fail(QTT_ERR_UNSUPPORTED, "qtt_batch_create: ranks above 48");
  }
  qtt_batch *B = new (std::nothrow) qtt_batch();
  if (!B) return fail(QTT_ERR_OOM, "qtt_batch_create: host allocation");
  B->ops.assign(ops, ops + nops);
  B->nrhs.assign(nrhs, nrhs + nops);
  B->ld.assign(ld, ld + nops);
  for (int i = 0; i < nops; ++i) {
    B->x.push_back(static_cast<const float *>(x[i]));
    B->y.push_back(static_cast<float *>(y[i]));
    B->flops += ops[i]->flops_per_rhs * (double)nrhs[i];
  }
  B->compute = compute;
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  B->budget = mem_budget ? mem_budget : std::min<size_t>(fr / 3, (size_t)64 << 30);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = persistent_alloc(reinterpret_cast<void **>(&B->d_status), sizeof(int), st) == QTT_OK
                      ? cudaSuccess : cudaErrorMemoryAllocation;
  if (e == cudaSuccess) e = cudaMemsetAsync(B->d_status, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    qtt_batch_destroy(B);
    return cuda_fail(e, "qtt_batch_create: status word");
  }
  qtt_status s = build_plan(B, st);
  if (s == QTT_OK) s = capture(B, st);
  if (s != QTT_OK) {
    qtt_batch_destroy(B);
    return s;
  }
  *out = B;
  return QTT_OK;
}

qtt_status qtt_batch_run(qtt_batch *B, void *stream) {
  if (!B || !B->exec) return fail(QTT_ERR_INVALID_ARG, "qtt_batch_run: no batch");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaGraphLaunch(B->exec, st);
  if (e != cudaSuccess) return cuda_fail(e, "qtt_batch_run: graph launch");
  for (int i : B->direct_ops) {
    const qtt_status s = apply_lp(B->ops[i], B->compute, B->x[i], QTT_F32, B->y[i], QTT_F32,
                                  B->nrhs[i], B->ld[i], st, LpEpilogue{});
    if (s != QTT_OK) return s;
  }
  // the run reads every operator and the batch's own buffers
  for (const qtt_op *A : B->ops) note_use(A, st);
  if (!B->last_run) {
    e = cudaEventCreateWithFlags(&B->last_run, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "qtt_batch_run: event");
  }
  e = cudaEventRecord(B->last_run, st);
  if (e != cudaSuccess) return cuda_fail(e, "qtt_batch_run: event record");
  return QTT_OK;
}

qtt_status qtt_batch_run_host(qtt_batch *B, const float *const *x_host, float *const *y_host,
                              void *stream) {
  if (!B || !B->exec) return fail(QTT_ERR_INVALID_ARG, "qtt_batch_run_host: no batch");
  if (!x_host || !y_host) return fail(QTT_ERR_INVALID_ARG, "qtt_batch_run_host: NULL array");
  const size_t nops = B->ops.size();
  for (size_t i = 0; i < nops; ++i)
    if (!x_host[i] || !y_host[i])
      return fail(QTT_ERR_INVALID_ARG, "qtt_batch_run_host: NULL vector");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CopyStreams cs;
  qtt_status s = copy_streams(&cs);
  if (s != QTT_OK) return s;
  cudaError_t e = cudaSuccess;
  const size_t nev = 4 + 2 * B->direct_ops.size();
  while (B->host_events.size() < nev && e == cudaSuccess) {
    cudaEvent_t ev = nullptr;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) B->host_events.push_back(ev);
  }
  if (e != cudaSuccess) return cuda_fail(e, "qtt_batch_run_host: events");
  cudaEvent_t *ev = B->host_events.data();
  std::vector<char> direct(nops, 0);
  for (int i : B->direct_ops) direct[i] = 1;
  // host rows are compact (leading dimension N); the batch's device vectors
  // have leading dimension ld
  auto copy_in = [&](size_t i) {
    const size_t row = ((size_t)1 << B->ops[i]->d) * sizeof(float);
    return cudaMemcpy2DAsync(const_cast<float *>(B->x[i]), (size_t)B->ld[i] * sizeof(float),
                             x_host[i], row, row, (size_t)B->nrhs[i], cudaMemcpyHostToDevice,
                             cs.in);
  };
  auto copy_out = [&](size_t i) {
    const size_t row = ((size_t)1 << B->ops[i]->d) * sizeof(float);
    return cudaMemcpy2DAsync(y_host[i], row, B->y[i], (size_t)B->ld[i] * sizeof(float), row,
                             (size_t)B->nrhs[i], cudaMemcpyDeviceToHost, cs.out);
  };
  // nothing starts before the work already on the caller's stream (an
  // earlier run may still read x or write y)
  e = cudaEventRecord(ev[0], st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs.in, ev[0], 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs.out, ev[0], 0);
  // the waves' inputs, the waves, their outputs
  for (size_t i = 0; i < nops && e == cudaSuccess; ++i)
    if (!direct[i]) e = copy_in(i);
  if (e == cudaSuccess) e = cudaEventRecord(ev[1], cs.in);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev[1], 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(B->exec, st);
  if (e == cudaSuccess) e = cudaEventRecord(ev[2], st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs.out, ev[2], 0);
  for (size_t i = 0; i < nops && e == cudaSuccess; ++i)
    if (!direct[i]) e = copy_out(i);
  // each direct operator: its input in, its apply, its output out
  for (size_t j = 0; j < B->direct_ops.size() && e == cudaSuccess && s == QTT_OK; ++j) {
    const int i = B->direct_ops[j];
    cudaEvent_t in_done = ev[4 + 2 * j], applied = ev[5 + 2 * j];
    e = copy_in(i);
    if (e == cudaSuccess) e = cudaEventRecord(in_done, cs.in);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, in_done, 0);
    if (e != cudaSuccess) break;
    s = apply_lp(B->ops[i], B->compute, B->x[i], QTT_F32, B->y[i], QTT_F32, B->nrhs[i],
                 B->ld[i], st, LpEpilogue{});
    if (s != QTT_OK) break;
    e = cudaEventRecord(applied, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs.out, applied, 0);
    if (e == cudaSuccess) e = copy_out(i);
  }
  // the caller's stream ends after the last copy out (also after an error)
  cudaError_t e2 = cudaEventRecord(ev[3], cs.out);
  if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(st, ev[3], 0);
  if (e2 != cudaSuccess) {
    cudaStreamSynchronize(cs.in);
    cudaStreamSynchronize(cs.out);
  }
  for (const qtt_op *A : B->ops) note_use(A, st);
  if (!B->last_run && cudaEventCreateWithFlags(&B->last_run, cudaEventDisableTiming) != cudaSuccess)
    return fail(QTT_ERR_CUDA, "qtt_batch_run_host: event");
  cudaEventRecord(B->last_run, st);
  if (s != QTT_OK) return s;
  if (e != cudaSuccess) return cuda_fail(e, "qtt_batch_run_host");
  if (e2 != cudaSuccess) return cuda_fail(e2, "qtt_batch_run_host: final ordering");
  return QTT_OK;
}

qtt_status qtt_batch_selftest_timeout(qtt_batch *B, double seconds, void *stream) {
  if (!B || B->waves.empty()) return fail(QTT_ERR_INVALID_ARG, "qtt_batch_selftest_timeout: no batch");
  if (!(seconds > 0.0 && seconds <= 10.0))
    return fail(QTT_ERR_INVALID_ARG, "qtt_batch_selftest_timeout: seconds must be in (0, 10]");
  if (B->waves[0].first_dep < 0)
    return fail(QTT_ERR_UNSUPPORTED,
                "qtt_batch_selftest_timeout: the first wave has no dependent items (every d = 1)");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, clk_khz = 2000000;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
  B->selftest_start = B->waves[0].first_dep;
  B->selftest_budget = (long long)(seconds * 1e3 * clk_khz);
  const qtt_status s = launch_waves(B, st);
  B->selftest_start = -1;
  B->selftest_budget = 0;
  for (const qtt_op *A : B->ops) note_use(A, st);
  if (!B->last_run && cudaEventCreateWithFlags(&B->last_run, cudaEventDisableTiming) != cudaSuccess)
    return fail(QTT_ERR_CUDA, "qtt_batch_selftest_timeout: event");
  cudaEventRecord(B->last_run, st);
  return s;
}

qtt_status qtt_batch_status(qtt_batch *B, void *stream) {
  if (!B) return fail(QTT_ERR_INVALID_ARG, "qtt_batch_status: no batch");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, B->d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "qtt_batch_status");
  if (h != 0) {
    cudaMemsetAsync(B->d_status, 0, sizeof(int), st);
    cudaStreamSynchronize(st);
    return fail(QTT_ERR_TIMEOUT, "batch kernel: a dependency wait ran out of its budget");
  }
  return QTT_OK;
}

qtt_status qtt_batch_set_variant(qtt_batch *B, int variant, void *stream) {
  if (!B) return fail(QTT_ERR_INVALID_ARG, "qtt_batch_set_variant: no batch");
  // variant = pairs per lane (2 or 4) + 100 x chunks per work item (1..64)
  // + 10000 x ring depth (2 or 3); missing parts mean 8 chunks and depth 3
  const int tn = variant % 100, sl = (variant / 100) % 100 ? (variant / 100) % 100 : 8;
  const int ns = variant / 10000 ? variant / 10000 : 3;
  if ((tn != 2 && tn != 4) || sl < 1 || sl > 64 || (ns != 2 && ns != 3))
    return fail(QTT_ERR_INVALID_ARG, "qtt_batch_set_variant: bad variant");
  B->variant = tn;
  B->slice = sl;
  B->stages = ns;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  QTT_CUDA_TRY(cudaStreamSynchronize(st));
  qtt_status s = build_plan(B, st);
  if (s == QTT_OK) s = capture(B, st);
  return s;
}

qtt_status qtt_batch_autotune(qtt_batch *B, int reps, void *stream, int *chosen,
                              double *seconds_per_run) {
  if (!B) return fail(QTT_ERR_INVALID_ARG, "qtt_batch_autotune: no batch");
  if (reps < 1) reps = 1;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int best = B->variant + 100 * B->slice + 10000 * B->stages;
  double best_t = 1e300;
  cudaEvent_t e0, e1;
  QTT_CUDA_TRY(cudaEventCreate(&e0));
  QTT_CUDA_TRY(cudaEventCreate(&e1));
  // no waves (every operator on the tensor-core path): nothing to tune, one
  // timed run reports the time
  const std::vector<int> cands =
      B->waves.empty() ? std::vector<int>{best} : std::vector<int>{30802, 33202, 33204, 23202, 23204};
  for (int v : cands) {
    qtt_status s = qtt_batch_set_variant(B, v, stream);
    if (s != QTT_OK) continue;
    qtt_batch_run(B, stream);  // warm-up
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps; ++r) qtt_batch_run(B, stream);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (qtt_batch_status(B, stream) != QTT_OK) continue;
    const double t = ms / 1e3 / reps;
    if (t < best_t) {
      best_t = t;
      best = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  qtt_status s = qtt_batch_set_variant(B, best, stream);
  if (chosen) *chosen = best;
  if (seconds_per_run) *seconds_per_run = best_t;
  return s;
}

qtt_status qtt_batch_direct_ops(const qtt_batch *B, int *count) {
  if (!B || !count) return fail(QTT_ERR_INVALID_ARG, "qtt_batch_direct_ops: no batch");
  *count = (int)B->direct_ops.size();
  return QTT_OK;
}

qtt_status qtt_batch_info(const qtt_batch *B, int *waves, int *variant, int *grid,
                          double *flops, size_t *scratch_bytes) {
  if (!B) return fail(QTT_ERR_INVALID_ARG, "qtt_batch_info: no batch");
  if (waves) *waves = (int)B->waves.size();
  if (variant) *variant = B->variant + 100 * B->slice + 10000 * B->stages;
  if (grid) *grid = B->grid;
  if (flops) *flops = B->flops;
  if (scratch_bytes) *scratch_bytes = B->scratch_bytes;
  return QTT_OK;
}

qtt_status qtt_batch_destroy(qtt_batch *B) {
  if (!B) return QTT_OK;
  // No device-wide synchronisation: the buffers go back to the pool after
  // the batch's last run (an in-flight graph is freed when it completes).
  free_waves(B);
  release(B, {B->scratch, B->d_next, B->d_status});
  if (B->last_run) cudaEventDestroy(B->last_run);
  for (cudaEvent_t ev : B->host_events) cudaEventDestroy(ev);  // released when complete
  delete B;
  return QTT_OK;
}

}  // extern "C"
