// Split-precision sample contraction on tcgen05 tensor cores (sm_103a).
//
// Computes, for each tile of 128 rows x 256 columns of a block's sums (Eq. 3),
//   C_b[r, c] += sum_s  A(s, r) B(s, c),   A = Y'_b,   B = w * [Y'_b | E Y'_b + Z_b]
// with Y' = Y - shift (first sweep: Y = O, Z = dE_L/dmu; second sweep: Y = p, Z = r of Eq. 6).
// Each FP32 operand value v is split as v = hi + lo:
//   BF16X4: hi = bf16(v), lo = bf16(v - hi) (v to 2^-17); hi*hi + hi*lo + lo*hi + lo*lo on
//           kind::f16 (lo is about 2^-9 v, so lo*lo is 2^-18 of the product and is kept);
//   TF32X4: hi = v to 8 bits, lo = tf32(v - hi) (v to 2^-21); the same four products on
//           kind::tf32.
// The operands are prepared once per element in HBM (blm_prep.cu) in the layout the tensor core
// reads -- one 128-byte row per parameter and sample group, [hi | lo] -- and this kernel only
// streams them: TMA (cp.async.bulk.tensor) into a shared-memory ring, tcgen05.mma into FP32
// accumulators in tensor memory, an epilogue that moves the accumulators into registers and, at
// the end of each work unit, into the FP64 sums with atomics.  Work units are (sample range,
// tile) pairs; a persistent grid of one CTA per SM walks them.
//
// Accumulation precision.  The tensor core adds each MMA's products into the FP32 accumulator
// with truncation toward zero, relative to the accumulator's magnitude: a term far smaller than
// the accumulator loses bits, always toward zero, and every accumulation shrinks the result by
// a fraction of an ulp.  Two measures keep the bias small (epilogue_split_role):
//  * the hi*hi products and the correction products go to separate accumulators, so the small
//    corrections meet an accumulator of their own size;
//  * the hi*hi accumulator runs in short intervals, each preloaded so that the values its
//    accumulations produce are centred on zero (centre_frac): the truncations of the negative
//    and positive halves cancel to first order.
// Every wait on an mbarrier is bounded; on timeout the kernel records an error code, drains the
// copies and MMAs it issued, frees tensor memory and returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "blm_internal.cuh"

namespace blm {

namespace {

constexpr int kBRows = 256;                       // B operand rows (output columns) per tile
constexpr int kARows = 128;                       // A operand rows (output rows) per tile
constexpr uint32_t kWaitLimit = 1u << 24;          // polls (each try_wait may suspend briefly)
// Stages per hi*hi accumulator interval (after the first stage of a unit, which is drained
// alone): 2, i.e. 64 samples (BF16) or 32 (TF32).  The tensor core truncates the terms it adds
// relative to the accumulator's magnitude, which grows with the interval; two stages keep the
// TF32 hi*hi products (22 significant bits) well above that grid, and the correction products
// of two stages (12 or 8 MMAs) cover the epilogue's drain of the interval before.
constexpr int kIntervalStages = 2;
constexpr int kMaxIntervalStages = kIntervalStages;
// Shortest sample range of a work unit (see the launchers).
constexpr int64_t kMinUnitSamples = 2048;

enum { A_VIEW = 0, A_SEPARATE = 1 };

struct Bars {
  uint64_t op_full[4];       // operand ring
  uint64_t op_empty[4];
  uint64_t db_full[2];       // prepared-operand kernel: [0] HH interval drained, [1] CR of a unit
  uint64_t db_empty[2];
  uint64_t drain;
  uint32_t tmem_base;
  int32_t abort;
  uint32_t wait_limit;       // polls of a pipeline wait before it gives up
};
static_assert(sizeof(Bars) <= 256, "barrier block exceeds its shared-memory slot");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ uint32_t mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok;
}

// Bounded wait: returns false (after recording `code`) if the phase never completes or another
// role has already aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, Bars* bars, int32_t* err,
                                          int code) {
  const uint32_t limit = bars->wait_limit;
  for (uint32_t i = 0; i < limit; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*(volatile int32_t*)&bars->abort) return false;
  }
  *(volatile int32_t*)&bars->abort = 1;
  atomicExch(err, code);
  return false;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of 128 bytes,
// 8-row groups 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);            // start address
  d |= (uint64_t)1u << 16;                           // leading byte offset (unused here)
  d |= (uint64_t)(1024u >> 4) << 32;                 // stride byte offset
  d |= (uint64_t)1u << 46;                           // version
  d |= (uint64_t)2u << 61;                           // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M = 128, N = 256.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((256u >> 3) << 17) |
                            ((128u >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}

// Instruction descriptor, kind::tf32: D = F32, A = B = TF32, both K-major, M = 128, N = 256.
constexpr uint32_t kIdescTf = (1u << 4) | (2u << 7) | (2u << 10) | ((256u >> 3) << 17) |
                              ((128u >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdescTf), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

#define TMEM_LD8(taddr, r)                                                                        \
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"          \
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),          \
                 "=r"(r[6]), "=r"(r[7])                                                           \
               : "r"(taddr))

#define TMEM_ST8(taddr, r)                                                                        \
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(   \
                   taddr),                                                                        \
               "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]),       \
               "r"(r[7])                                                                          \
               : "memory")

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

struct TileInfo {
  int a_map, b_map, a_row, b_row, nA, nB, amode, packed;
  double* out;
  int64_t out_ld;
};

__device__ __forceinline__ TileInfo decode_tile(const TcTile& t, bool weighted) {
  TileInfo ti;
  ti.a_map = t.a_map;
  ti.b_map = t.b_map;
  ti.a_row = t.a_row;
  ti.b_row = t.b_row;
  ti.nA = t.nA;
  ti.nB = t.nB;
  ti.amode = (t.a_view && !weighted) ? A_VIEW : A_SEPARATE;
  ti.packed = t.packed;
  ti.out = t.out;
  ti.out_ld = t.out_ld;
  return ti;
}

// Tensor maps of the operand arrays of one launch: boxes of 256 rows (B) and 128 rows (A).
struct OpMaps {
  CUtensorMap b[kTcMaps];
  CUtensorMap a[kTcMaps];
};

struct Params {
  int weighted;          // the B operand rows carry sample weights (A is then never a view)
  TcPack pack;           // block tables of packed tiles
  int64_t ns;
  const TcTile* tiles;
  int ntiles;
  int64_t range_len;     // samples per unit (multiple of the stage)
  int64_t nunits;
  int flush_stages;
  int32_t* err;
  uint32_t wait_limit;   // polls of a pipeline wait (mbarrier) before the kernel gives up
};

// Accumulator intervals of a unit with nst stages: interval 0 is stage 0 alone, interval i >= 1
// covers stages 1 + (i - 1) fs .. min(nst, 1 + i fs) - 1.
__device__ __forceinline__ int interval_count(int nst, int fs) {
  return nst <= 1 ? 1 : 1 + (nst - 1 + fs - 1) / fs;
}
__device__ __forceinline__ int interval_len(int i, int nst, int fs) {
  return i == 0 ? 1 : min(fs, nst - 1 - (i - 1) * fs);
}
// Where the preload puts the accumulator.  An interval of q K-steps (q hi*hi products, each
// followed by its correction products at about the same value) takes the accumulator from d to
// d + P in q equal increments, and every accumulation truncates relative to the value it
// produces: the q levels d + P/q, .., d + P average d + P (q + 1) / (2 q).  Starting at
// d = -P (q + 1) / (2 q) centres them on zero, so the truncations of the negative and positive
// halves cancel to first order.  Returns (q + 1) / (2 q).
__device__ __forceinline__ float centre_frac(int q) { return 0.5f + 0.5f / (float)q; }

// Samples per operand stage of the TMA-fed kernel: one 128-byte row per parameter, two K steps
// per row half -- BF16: 32 samples (K = 16), TF32: 16 samples (K = 8).
template <bool TF>
__device__ __host__ constexpr int op_stage_k() { return TF ? 16 : 32; }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// ---------------------------------------------------------------------------------------------
// Split accumulation for tc_op_kernel.  Tensor memory holds two 256-column FP32 accumulators:
//   HH (columns 0-255)   the hi*hi products, in preloaded intervals of kIntervalStages stages;
//   CR (columns 256-511) the correction products hi*lo + lo*hi + lo*lo of the whole work unit.
// The tensor core aligns the terms of every accumulation to the accumulator's magnitude and
// truncates the bits below that grid, so a product far smaller than the accumulator loses a
// fraction of itself, always toward zero.  The corrections are 2^-8 (hi*lo, lo*hi) and 2^-16
// (lo*lo) of the hi*hi terms; added into the large HH accumulator, the lo*lo terms -- positive on
// the diagonal of every overlap block -- were partly cut off, a bias of about -3e-7 relative on
// the diagonal of S_b.  In CR they meet an accumulator of their own size (hi*lo and lo*hi have
// random signs, so CR stays near 2^-8 sqrt(N) of a single product), where the grid is fine.
//
// HH: interval 0 (the first stage alone) starts from zero, interval i >= 1 from a preload d_i of
// about -(q + 1) / (2 q) of the partial sum it is expected to add (q = its K-steps, centre_frac),
// written into the buffer by the epilogue when it drains interval i - 1.  The epilogue keeps, in
// registers, U = sum of drained values - sum of written preloads; since every preload is drained
// before the next is written, U + V at the drain of interval i is the exact running total s,
// d_{i+1} = kappa_i s with kappa_i = -(q + 1) / (2 q) len(i + 1) / stages_through(i), and
// U <- s - d_{i+1}.  After the unit's last drain U is the hi*hi sum; CR is then added once.
// The MMA warp issues the correction products of all of an interval's stages before its hi*hi
// products, so that while the epilogue drains HH at an interval boundary the tensor pipe works
// on CR.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ int stages_through(int i, int nst, int fs) {
  return i == 0 ? 1 : min(nst, 1 + i * fs);
}
// Two K-steps (of 16 samples) per 32-sample stage: an interval of len stages has 2 len levels.
__device__ __forceinline__ float split_kappa(int i, int nst, int fs) {
  const int len = interval_len(i + 1, nst, fs);
  return -centre_frac(2 * len) * (float)len / (float)stages_through(i, nst, fs);
}

template <bool TF>
__device__ __forceinline__ void epilogue_split_role(const Params& P, Bars* bars, uint32_t tmem,
                                                    int warp, int lane, int fs) {
  constexpr int kTmaStageK = op_stage_k<TF>();
  const int q = warp & 3;                          // tensor-memory lane quadrant
  const int h = (warp - 2) >> 2;                   // warps 2-5: columns 0-127, 6-9: 128-255
  const uint32_t lane_addr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(128 * h);
  const int row = 32 * q + lane;
  uint32_t k = 0, j = 0;
  bool alive = true;
  float U[128];
  for (int64_t u = blockIdx.x; u < P.nunits && alive; u += gridDim.x, ++j) {
    const int64_t sa = (u / P.ntiles) * P.range_len;
    const int64_t sb = min(P.ns, sa + P.range_len);
    const int nst = (int)((sb - sa + kTmaStageK - 1) / kTmaStageK);
    const int nint = interval_count(nst, fs);
#pragma unroll
    for (int i = 0; i < 128; ++i) U[i] = 0.0f;
    for (int it = 0; it < nint; ++it, ++k) {
      alive = mbar_wait(&bars->db_full[0], k & 1, bars, P.err, 13);
      if (!alive) break;
      tc_fence_after();
      const bool pre = it + 1 < nint;
      const float kap = pre ? split_kappa(it, nst, fs) : 0.0f;
#pragma unroll
      for (int c = 0; c < 16; c += 2) {
        uint32_t a[8], b[8];
        TMEM_LD8(lane_addr + 8 * c, a);
        TMEM_LD8(lane_addr + 8 * c + 8, b);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float s = U[8 * c + i] + __uint_as_float(a[i]);
          const float d = kap * s;
          U[8 * c + i] = s - d;
          a[i] = __float_as_uint(d);
          const float s1 = U[8 * c + 8 + i] + __uint_as_float(b[i]);
          const float d1 = kap * s1;
          U[8 * c + 8 + i] = s1 - d1;
          b[i] = __float_as_uint(d1);
        }
        if (pre) {
          TMEM_ST8(lane_addr + 8 * c, a);
          TMEM_ST8(lane_addr + 8 * c + 8, b);
        }
      }
      if (pre) tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars->db_empty[0]);
    }
    if (!alive) break;
    // the unit's corrections
    alive = mbar_wait(&bars->db_full[1], j & 1, bars, P.err, 16);
    if (!alive) break;
    tc_fence_after();
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      uint32_t a[8];
      TMEM_LD8(lane_addr + 256 + 8 * c, a);
      tmem_wait_ld();
#pragma unroll
      for (int i = 0; i < 8; ++i) U[8 * c + i] += __uint_as_float(a[i]);
    }
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&bars->db_empty[1]);
    const TileInfo ti = decode_tile(P.tiles[u % P.ntiles], P.weighted != 0);
    if (row < ti.nA && !ti.packed) {
      double* orow = ti.out + (int64_t)row * ti.out_ld + 128 * h;
      const int ncol = min(128, ti.nB - 128 * h);
#pragma unroll
      for (int i = 0; i < 128; ++i)
        if (i < ncol) atomicAdd(orow + i, (double)U[i]);
    } else if (row < ti.nA) {
      // band tile: this row's block keeps the columns of the same block
      const int64_t r = ti.a_row + row;
      const int b = P.pack.blk_of[r];
      const int64_t lo = P.pack.lo[b];
      const int m = P.pack.m[b];
      const int64_t c0 = ti.b_row + 128 * h;
      const int i_lo = (int)max((int64_t)0, lo - c0);
      const int i_hi = (int)min(min((int64_t)128, lo + m - c0), (int64_t)(ti.nB - 128 * h));
      double* orow = P.pack.C[b] + (r - lo) * 2 * m + (c0 - lo) + (ti.b_map == 2 ? m : 0);
#pragma unroll
      for (int i = 0; i < 128; ++i)
        if (i >= i_lo && i < i_hi) atomicAdd(orow + i, (double)U[i]);
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Prepared-operand variant (BF16X4): the operands were written to HBM once per sweep by the
// preparation kernel (blm_prep.cu) in the tensor core's layout -- one 128-byte row per parameter
// and 32-sample group holding [hi(32) | lo(32)] -- so this kernel only streams them: warp 1 loads
// each stage's B rows (256 x 128 bytes) and, unless A is a view of B, its A rows (128 x 128
// bytes) with 128-byte-swizzled cp.async.bulk.tensor into a four-deep ring; warp 0 issues the
// products of two K steps into the HH and CR accumulators; warps 2-9 are the epilogue
// (epilogue_split_role).  No converter warps.
// ---------------------------------------------------------------------------------------------
constexpr int kOpStagesP = 4;
constexpr int kPStageBytes = (kBRows + kARows) * 128;          // 48 KB
constexpr int kPBarOffset = kOpStagesP * kPStageBytes;          // 192 KB
constexpr int kPSmemBytes = kPBarOffset + 256 + 1024;
constexpr int kPThreads = 320;           // MMA, TMA, eight epilogue warps
static_assert(kPSmemBytes <= 227 * 1024, "prepared-operand kernel exceeds shared memory");

template <bool TF>
__global__ void __maxnreg__(168)
tc_op_kernel(const Params P, const __grid_constant__ OpMaps maps) {
  constexpr int kTmaStageK = op_stage_k<TF>();
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  Bars* bars = (Bars*)(smem + kPBarOffset);
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kOpStagesP; ++s) {
      mbar_init(&bars->op_full[s], 1);
      mbar_init(&bars->op_empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bars->db_full[b], 1);
      mbar_init(&bars->db_empty[b], 8);
    }
    mbar_init(&bars->drain, 1);
    bars->abort = 0;
    bars->wait_limit = P.wait_limit;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_u32(&bars->tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem_base;
  const int fs = P.flush_stages;

  if (warp == 0) {
    // ------------------------------- MMA issuer -------------------------------
    uint32_t g = 0, k = 0, j = 0;
    bool alive = true;
    for (int64_t u = blockIdx.x; u < P.nunits && alive; u += gridDim.x, ++j) {
      const TileInfo ti = decode_tile(P.tiles[u % P.ntiles], P.weighted != 0);
      const int64_t sa = (u / P.ntiles) * P.range_len;
      const int64_t sb = min(P.ns, sa + P.range_len);
      const int nst = (int)((sb - sa + kTmaStageK - 1) / kTmaStageK);
      // interval by interval (stage 0 alone, then fs stages): every stage's correction
      // products first -- they keep the tensor pipe busy while the epilogue drains HH -- then,
      // once the previous interval's drain is complete, the interval's hi*hi products
      const int nint = interval_count(nst, fs);
      for (int it = 0, st0 = 0; it < nint && alive; ++it) {
        const int len = interval_len(it, nst, fs);
        uint32_t ob[kMaxIntervalStages], oa[kMaxIntervalStages], slot[kMaxIntervalStages];
#pragma unroll
        for (int q = 0; q < kMaxIntervalStages; ++q) {
          if (q >= len || !alive) break;
          const int st = st0 + q;
          const uint32_t gq = g + (uint32_t)q;
          slot[q] = gq % kOpStagesP;
          if (st == 0) {
            // the unit's first correction product overwrites CR: the previous unit's CR must
            // have been read
            alive = mbar_wait(&bars->db_empty[1], (j & 1) ^ 1, bars, P.err, 17);
            tc_fence_after();
          }
          if (alive) alive = mbar_wait(&bars->op_full[slot[q]], (gq / kOpStagesP) & 1, bars, P.err, 12);
          if (!alive) break;
          tc_fence_after();
          ob[q] = smem_u32(smem + slot[q] * kPStageBytes);
          oa[q] = (ti.amode == A_VIEW) ? ob[q] + (uint32_t)(ti.a_row - ti.b_row) * 128u
                                       : ob[q] + (uint32_t)kBRows * 128u;
          if (lane == 0) {
            // lo is about 2^-9 of hi in both splits, so lo * lo (2^-18) is kept
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
              const uint32_t o = ks * 32;
              const uint32_t a0 = (st == 0 && ks == 0) ? 0u : 1u;
              if (TF) {
                mma_tf32(tmem + 256u, sdesc(oa[q] + o), sdesc(ob[q] + 64 + o), a0);       // hi * lo
                mma_tf32(tmem + 256u, sdesc(oa[q] + 64 + o), sdesc(ob[q] + o), 1);        // lo * hi
                mma_tf32(tmem + 256u, sdesc(oa[q] + 64 + o), sdesc(ob[q] + 64 + o), 1);   // lo * lo
              } else {
                mma_bf16(tmem + 256u, sdesc(oa[q] + o), sdesc(ob[q] + 64 + o), a0);       // hi * lo
                mma_bf16(tmem + 256u, sdesc(oa[q] + 64 + o), sdesc(ob[q] + o), 1);        // lo * hi
                mma_bf16(tmem + 256u, sdesc(oa[q] + 64 + o), sdesc(ob[q] + 64 + o), 1);   // lo * lo
              }
            }
          }
          __syncwarp();
        }
        if (!alive) break;
        // interval 0 of a unit starts HH from zero, later intervals from the epilogue's
        // preload: either way the previous interval's drain must be complete
        alive = mbar_wait(&bars->db_empty[0], (k & 1) ^ 1, bars, P.err, 11);
        tc_fence_after();
        uint32_t acc = (it == 0) ? 0u : 1u;
        if (lane == 0) {
#pragma unroll
          for (int q = 0; q < kMaxIntervalStages; ++q) {
            if (q >= len) break;
            if (alive) {
#pragma unroll
              for (int ks = 0; ks < 2; ++ks) {
                if (TF)
                  mma_tf32(tmem, sdesc(oa[q] + ks * 32), sdesc(ob[q] + ks * 32), acc);   // hi * hi
                else
                  mma_bf16(tmem, sdesc(oa[q] + ks * 32), sdesc(ob[q] + ks * 32), acc);   // hi * hi
                acc = 1;
              }
            }
            mma_commit(&bars->op_empty[slot[q]]);
          }
          if (alive) mma_commit(&bars->db_full[0]);
          if (alive && it == nint - 1) mma_commit(&bars->db_full[1]);
        }
        __syncwarp();
        g += (uint32_t)len;
        st0 += len;
        ++k;
      }
    }
    if (lane == 0) mma_commit(&bars->drain);
    __syncwarp();
    for (uint32_t i = 0; i < kWaitLimit && !mbar_try_wait(&bars->drain, 0); ++i) {
    }
  } else if (warp == 1) {
    // ------------------------------- TMA producer ------------------------------
    uint32_t g = 0;
    uint32_t armed[kOpStagesP] = {0, 0, 0, 0};
    bool alive = true;
    for (int64_t u = blockIdx.x; u < P.nunits && alive; u += gridDim.x) {
      const TileInfo ti = decode_tile(P.tiles[u % P.ntiles], P.weighted != 0);
      const int64_t sa = (u / P.ntiles) * P.range_len;
      const int64_t sb = min(P.ns, sa + P.range_len);
      const int nst = (int)((sb - sa + kTmaStageK - 1) / kTmaStageK);
      const bool aview = ti.amode == A_VIEW;
      const uint32_t bytes = (uint32_t)kBRows * 128u + (aview ? 0u : (uint32_t)kARows * 128u);
      const CUtensorMap* mb = &maps.b[ti.b_map];
      for (int st = 0; st < nst && alive; ++st, ++g) {
        const uint32_t slot = g % kOpStagesP, use = g / kOpStagesP;
        alive = mbar_wait(&bars->op_empty[slot], (use & 1) ^ 1, bars, P.err, 15);
        if (!alive) break;
        if (lane == 0) {
          uint64_t* bar = &bars->op_full[slot];
          const uint32_t dst = smem_u32(smem + slot * kPStageBytes);
          const int x = (int)((sa / kTmaStageK + st) * 64);
          mbar_expect_tx(bar, bytes);
          tma_load_2d(dst, mb, x, ti.b_row, bar);
          if (!aview) tma_load_2d(dst + kBRows * 128, &maps.a[ti.a_map], x, ti.a_row, bar);
        }
        __syncwarp();
        armed[slot] = use + 1;
      }
    }
    for (int s = 0; s < kOpStagesP; ++s)
      if (armed[s] > 0) {
        for (uint32_t i = 0; i < kWaitLimit && !mbar_try_wait(&bars->op_full[s], (armed[s] - 1) & 1);
             ++i) {
        }
      }
  } else if (warp >= 2 && warp < 10) {
    epilogue_split_role<TF>(P, bars, tmem, warp, lane, fs);
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem)
                 : "memory");
  }
}

}  // namespace

namespace {
// cuTensorMapEncodeTiled, looked up through the runtime (no link-time dependence on the driver
// library, so that the library still loads on machines without a GPU driver).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

}  // namespace

namespace {
// 2-D tensor map over prepared bf16 operand rows: nrows x (row_bytes / 2) elements, boxes of
// 64 elements (128 bytes) x box_rows rows, 128-byte swizzle (the layout tcgen05 reads K-major).
bool encode_op_map(CUtensorMap* m, const uint8_t* base, int64_t nrows, int64_t row_bytes,
                   int box_rows) {
  EncodeTiledFn fn = encode_tiled_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)(row_bytes / 2), (cuuint64_t)nrows};
  cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
  cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint8_t*>(base), dims, strides,
            box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace

cudaError_t launch_tc_prepared(const TcOperands& ops, int64_t row_bytes, int64_t ns,
                               const TcTile* tiles, int ntiles, int weighted, int32_t* err,
                               uint32_t wait_limit, int tf32, const TcPack& pack,
                               int64_t max_range, cudaStream_t st) {
  if (ns <= 0 || ntiles <= 0) return cudaSuccess;
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(tc_op_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPSmemBytes);
    cudaFuncSetAttribute(tc_op_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPSmemBytes);
  }
  const int stage = tf32 ? op_stage_k<true>() : op_stage_k<false>();
  OpMaps maps;
  for (int i = 0; i < kTcMaps; ++i) {
    // unused slots repeat the first array (never addressed by a tile)
    const uint8_t* base = ops.op[i] ? ops.op[i] : ops.op[0];
    const int64_t rows = ops.op[i] ? ops.rows[i] : ops.rows[0];
    if (!encode_op_map(&maps.b[i], base, rows, row_bytes, kBRows) ||
        !encode_op_map(&maps.a[i], base, rows, row_bytes, kARows))
      return cudaErrorInvalidValue;
  }
  Params P;
  P.weighted = weighted;
  P.pack = pack;
  P.ns = ns;
  P.tiles = tiles;
  P.ntiles = ntiles;
  // sample ranges of up to max_range: each unit ends in one flush of its sums with FP64 atomics
  // and one wait for the drain of its last interval, so units are kept long; at least four
  // units per SM keep the tail short, and no unit is shorter than kMinUnitSamples
  int64_t range = max_range > kMinUnitSamples ? max_range : kMinUnitSamples;
  while (range > kMinUnitSamples && ((ns + range - 1) / range) * ntiles < 4LL * sms) range /= 2;
  P.range_len = range;
  P.nunits = ((ns + range - 1) / range) * ntiles;
  P.flush_stages = kIntervalStages;
  (void)stage;
  P.err = err;
  P.wait_limit = wait_limit;
  const int grid = (int)(P.nunits < sms ? P.nunits : sms);
  if (tf32)
    tc_op_kernel<true><<<grid, kPThreads, kPSmemBytes, st>>>(P, maps);
  else
    tc_op_kernel<false><<<grid, kPThreads, kPSmemBytes, st>>>(P, maps);
  return cudaGetLastError();
}

}  // namespace blm
