// Split-BF16 sample contraction on tcgen05 tensor cores (sm_103a).
//
// Computes, for each tile of 128 rows x 256 columns of a block's sums (Eq. 3),
//   C_b[r, c] += sum_s  A(s, r) B(s, c),   A = Y'_b,   B = w * [Y'_b | E Y'_b + Z_b]
// with Y' = Y - shift (first sweep: Y = O, Z = dE_L/dmu; second sweep: Y = p, Z = r of Eq. 6).
// Each FP32 operand value v is split as v = hi + lo + O(2^-16 v) with hi = bf16(v),
// lo = bf16(v - hi); the four products hi*hi + hi*lo + lo*hi + lo*lo are accumulated by
// tcgen05.mma (kind::f16, BF16 inputs, FP32 accumulator in tensor memory).  lo is about 2^-8 v
// (bf16 keeps 8 significant bits), so lo*lo is 2^-16 of the product and cannot be dropped.
//
// Accumulation precision.  The tensor core adds each MMA's products into the FP32 accumulator
// with truncation (round toward zero): every accumulation shrinks |D| by up to one ulp, a bias of
// about 2^-25 |D| per accumulation that does not average out (measured: -6e-7 relative on the
// diagonal sums after 16 accumulations).  Two measures keep it small:
//  * the tensor-memory accumulator (L1, 256 columns) runs for short intervals -- the first
//    stage of a unit alone, then `flush_stages` stages -- after which the epilogue warps add it
//    into a second FP32 accumulator in tensor memory (L2, 256 columns, round-to-nearest CUDA-core
//    adds), and at the end of each work unit add L2 + L1 into the FP64 result with atomics;
//  * L1 does not restart from zero: the epilogue preloads it with minus (q + 1) / (2 q) of the
//    partial sum P the interval is expected to add (q = its K-steps; the expectation is the
//    running per-stage mean in L2 times the interval length), so the values the accumulations
//    produce are centred on zero and the truncations of the negative and positive halves cancel
//    to first order (centre_frac).  The preloaded value is recomputed bit for bit from L2 when
//    the interval is flushed and subtracted exactly.
// Work units are (sample range, tile) pairs; a persistent grid of one CTA per SM walks them.
//
// Two kernels.  tc_op_kernel (the BF16X4 path) streams operand rows prepared once per element
// by blm_prep.cu with TMA and keeps two tensor-memory accumulators that alternate per interval,
// the running sums in epilogue registers (described at the kernel).  tc_accumulate_kernel (the
// TF32X3 path, or where operands are not prepared) converts FP32 samples in the kernel and uses
// the L1 / L2 scheme above: warp 0 allocates tensor memory and one lane issues the MMAs; warps
// 4-7 are the epilogue (one per 32-lane tensor-memory quadrant); the other 11 warps convert
// FP32 samples into the split operands in shared memory (K-major, 128-byte swizzle: each operand
// row holds 64 consecutive samples of one parameter).
// Every wait on an mbarrier is bounded; on timeout the kernel records an error code, drains its
// own MMAs, frees tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "blm_internal.cuh"

namespace blm {

namespace {

constexpr int kWarps = 16;
constexpr int kThreads = kWarps * 32;
constexpr int kStageK = 64;                       // samples per stage (BF16 operands)
constexpr int kStageKTf = 32;                     // samples per stage (TF32 operands)
template <bool TF>
__device__ __host__ constexpr int stage_k() { return TF ? kStageKTf : kStageK; }
constexpr int kStages = 2;
constexpr int kBRows = 256;
constexpr int kARows = 128;
constexpr int kBBytes = kBRows * 128;             // one split half of B: 32 KB
constexpr int kABytes = kARows * 128;             // one split half of A: 16 KB
constexpr int kStageBytes = 2 * kBBytes + 2 * kABytes;
constexpr int kConvWarps = 11;
constexpr int kBarOffset = kStages * kStageBytes;
constexpr int kSmemBytes = kBarOffset + 256 + 1024;   // + barriers + alignment slack
constexpr uint32_t kWaitLimit = 1u << 24;          // polls (each try_wait may suspend briefly)
// Samples per tensor-memory accumulator interval (after the first stage of a unit, which is
// flushed alone): 128, i.e. 32 accumulations of the four split products.
constexpr int kFlushSamples = 128;
// Shortest sample range of a work unit (see the launchers).
constexpr int64_t kMinUnitSamples = 2048;

enum { A_VIEW = 0, A_FROM_B = 1, A_SEPARATE = 2 };

struct Bars {
  uint64_t op_full[4];       // operand ring (kStages slots, four in tc_op_kernel)
  uint64_t op_empty[4];
  uint64_t l1_full;
  uint64_t l1_empty;
  uint64_t db_full[2];       // prepared-operand kernel: [0] HH interval drained, [1] CR of a unit
  uint64_t db_empty[2];
  uint64_t drain;
  uint32_t tmem_base;
  int32_t abort;
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
  for (uint32_t i = 0; i < kWaitLimit; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*(volatile int32_t*)&bars->abort) return false;
  }
  *(volatile int32_t*)&bars->abort = 1;
  atomicExch(err, code);
  return false;
}

__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
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

#define TMEM_LD32(taddr, r)                                                                       \
  asm volatile(                                                                                   \
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"    \
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"          \
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),       \
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),   \
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),            \
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),            \
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])             \
      : "r"(taddr))

#define TMEM_ST32(taddr, r)                                                                       \
  asm volatile(                                                                                   \
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13," \
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(     \
          taddr),                                                                                 \
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),     \
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),          \
      "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]),        \
      "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]),        \
      "r"(r[29]), "r"(r[30]), "r"(r[31])                                                          \
      : "memory")

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

#define TMEM_LD16(taddr, r)                                                                       \
  asm volatile(                                                                                   \
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"    \
      "%14,%15}, [%16];"                                                                          \
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),       \
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),   \
        "=r"(r[14]), "=r"(r[15])                                                                  \
      : "r"(taddr))

#define TMEM_ST16(taddr, r)                                                                       \
  asm volatile(                                                                                   \
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13," \
      "%14,%15,%16};" ::"r"(taddr),                                                               \
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),     \
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),          \
      "r"(r[15])                                                                                  \
      : "memory")

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// bf16x2 packing: the first element goes to the low half (lower address).
__device__ __forceinline__ uint32_t pack2(float first, float second) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(second), "f"(first));
  return d;
}

// Split 8 values into hi/lo bf16 (4 words each).
__device__ __forceinline__ void split8(const float* v, uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t hh = pack2(v[2 * k], v[2 * k + 1]);
    const float h0 = __uint_as_float(hh << 16);
    const float h1 = __uint_as_float(hh & 0xFFFF0000u);
    h[k] = hh;
    l[k] = pack2(v[2 * k] - h0, v[2 * k + 1] - h1);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Operand stores carry no "memory" clobber so that the next job's global loads can be hoisted
// above them; the proxy fence before the mbarrier arrive orders them for the tensor core.
// Split 8 values into TF32 hi (round to nearest) and FP32 lo = v - hi (exact); the tensor core
// reads lo's top 19 bits, so hi + lo represents v to 2^-22 relative.  Two 16-byte chunks each.
__device__ __forceinline__ void split8_tf32(const float* v, uint4* hi, uint4* lo) {
  uint32_t h[8], l[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    uint32_t t;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(v[k]));
    h[k] = t;
    l[k] = __float_as_uint(v[k] - __uint_as_float(t));
  }
  hi[0] = make_uint4(h[0], h[1], h[2], h[3]);
  hi[1] = make_uint4(h[4], h[5], h[6], h[7]);
  lo[0] = make_uint4(l[0], l[1], l[2], l[3]);
  lo[1] = make_uint4(l[4], l[5], l[6], l[7]);
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint4 v) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y),
               "r"(v.z), "r"(v.w));
}

// Byte offset of (row, 16-byte chunk) in a K-major 128-byte-swizzled operand tile.
__device__ __forceinline__ uint32_t swz(int row, int chunk) {
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((chunk ^ (row & 7)) << 4));
}

struct TileInfo {
  int64_t lo;
  int m, row0, col0, pb, nB, nA, xtype, amode;
  double* out;
};

// A is a view of B's rows only when both hold the same unweighted Y' values.
__device__ __forceinline__ TileInfo decode_tile(const TcTile& t, bool weighted) {
  TileInfo ti;
  ti.lo = t.lo;
  ti.m = t.m;
  ti.row0 = t.row0;
  ti.col0 = t.col0;
  ti.out = t.out;
  ti.xtype = t.col0 >= t.m;
  ti.pb = ti.xtype ? t.col0 - t.m : t.col0;
  ti.nB = min(kBRows, (ti.xtype ? 2 * t.m : t.m) - t.col0);
  ti.nA = min(kARows, t.m - t.row0);
  if (!weighted && !ti.xtype && ti.pb <= ti.row0 && ti.row0 + kARows <= ti.pb + kBRows)
    ti.amode = A_VIEW;
  else if (ti.xtype && ti.pb <= ti.row0 && ti.row0 + kARows <= ti.pb + ti.nB)
    ti.amode = A_FROM_B;
  else
    ti.amode = A_SEPARATE;
  return ti;
}

struct Params {
  const float* Y;
  const float* Z;
  const float* E;
  const float* w;
  const float* shift;
  int64_t ns;
  int64_t ld;
  const TcTile* tiles;
  int ntiles;
  int64_t range_len;     // samples per unit (multiple of kStageK)
  int64_t nunits;
  int flush_stages;
  int vec_ok;            // base pointers 16-byte aligned and ld a multiple of 4
  int32_t* err;
};

// Converter job: 32 operand rows x 32 samples (8 sample groups g of 8, lane = 8 g + l).
// VEC: lane l owns rows 4l .. 4l+3 and loads them as float4 (needs 16-byte aligned rows);
// otherwise lane l owns rows l + 8e with scalar loads.  Both orders give conflict-free 16-byte
// swizzled stores.  All loads of a job are issued before any value is used.
// kind 0: B rows (Y' or X', weighted; A rows too in A_FROM_B mode); kind 1: A rows (Y').
template <bool VEC, bool TF>
__device__ __forceinline__ void convert_job(const Params& P, const TileInfo& ti, int kind,
                                            int rowgroup, int half, int64_t stage_base,
                                            int64_t s_end, uint8_t* stage) {
  const int lane = threadIdx.x & 31;
  const int g = lane >> 3, l = lane & 7;
  const int64_t s0 = stage_base + 32 * half + 8 * g;
  const bool xt = (kind == 0) && ti.xtype;
  float ev[8], wv[8];
  bool vs[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int64_t s = s0 + q;
    vs[q] = s < s_end;
    ev[q] = (xt && vs[q]) ? __ldg(P.E + s) : 0.0f;
    wv[q] = (kind == 0 && P.w && vs[q]) ? __ldg(P.w + s) : 1.0f;
  }
  int row[4];
  int64_t par[4];
  bool vr[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    row[e] = rowgroup * 32 + (VEC ? 4 * l + e : l + 8 * e);
    if (kind == 0) {
      vr[e] = row[e] < ti.nB;
      par[e] = ti.lo + ti.pb + row[e];
    } else {
      vr[e] = row[e] < ti.nA;
      par[e] = ti.lo + ti.row0 + row[e];
    }
  }
  float y[4][8], z[4][8];
  if (VEC) {
    // rows 4l .. 4l+3 are all valid or all invalid: nB and nA are multiples of 4 here
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      float4 a = make_float4(0.f, 0.f, 0.f, 0.f), c = a;
      if (vr[0] && vs[q]) {
        const int64_t idx = (s0 + q) * P.ld + par[0];
        a = __ldg(reinterpret_cast<const float4*>(P.Y + idx));
        if (xt) c = __ldg(reinterpret_cast<const float4*>(P.Z + idx));
      }
      y[0][q] = a.x; y[1][q] = a.y; y[2][q] = a.z; y[3][q] = a.w;
      z[0][q] = c.x; z[1][q] = c.y; z[2][q] = c.z; z[3][q] = c.w;
    }
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e)
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const bool ok = vr[e] && vs[q];
        const int64_t idx = (s0 + q) * P.ld + par[e];
        y[e][q] = ok ? __ldg(P.Y + idx) : 0.0f;
        z[e][q] = (ok && xt) ? __ldg(P.Z + idx) : 0.0f;
      }
  }
  // BF16: one 16-byte chunk of 8 samples per row; TF32: two chunks of 4 samples
  const int chunk = TF ? 2 * g : 4 * half + g;
  const uint32_t sbase = smem_u32(stage);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float sh = (vr[e] && P.shift) ? __ldg(P.shift + par[e]) : 0.0f;
    float yy[8], x[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const bool ok = vr[e] && vs[q];
      yy[q] = ok ? y[e][q] - sh : 0.0f;
      x[q] = (xt ? fmaf(ev[q], yy[q], z[e][q]) : yy[q]) * wv[q];
    }
    const uint32_t off = swz(row[e], chunk);
    const int arow = ti.pb + row[e] - ti.row0;
    const bool a_from_b = (kind == 0) && (ti.amode == A_FROM_B) && arow >= 0 && arow < kARows;
    const uint32_t aoff = swz(kind == 0 ? arow : row[e], chunk);
    if (TF) {
      uint4 hi[2], lo[2];
      const uint32_t off1 = swz(row[e], chunk + 1);
      if (kind == 0) {
        split8_tf32(x, hi, lo);
        st_shared_v4(sbase + off, hi[0]);
        st_shared_v4(sbase + off1, hi[1]);
        st_shared_v4(sbase + kBBytes + off, lo[0]);
        st_shared_v4(sbase + kBBytes + off1, lo[1]);
      }
      if (kind == 1 || a_from_b) {
        split8_tf32(yy, hi, lo);
        const uint32_t aoff1 = swz(kind == 0 ? arow : row[e], chunk + 1);
        st_shared_v4(sbase + 2 * kBBytes + aoff, hi[0]);
        st_shared_v4(sbase + 2 * kBBytes + aoff1, hi[1]);
        st_shared_v4(sbase + 2 * kBBytes + kABytes + aoff, lo[0]);
        st_shared_v4(sbase + 2 * kBBytes + kABytes + aoff1, lo[1]);
      }
    } else {
      uint4 hi, lo;
      if (kind == 0) {
        split8(x, hi, lo);
        st_shared_v4(sbase + off, hi);
        st_shared_v4(sbase + kBBytes + off, lo);
      }
      if (kind == 1 || a_from_b) {
        split8(yy, hi, lo);
        st_shared_v4(sbase + 2 * kBBytes + aoff, hi);
        st_shared_v4(sbase + 2 * kBBytes + kABytes + aoff, lo);
      }
    }
  }
}

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

// Preload factor of interval i >= 1 (kq K-steps per stage): L1 starts at coef * L2, L2 holding
// the sum of the previous stages_done = 1 + (i - 1) fs stages.
__device__ __forceinline__ float preload_coef(int i, int nst, int fs, int kq) {
  const int len = interval_len(i, nst, fs);
  return -centre_frac(kq * len) * (float)len / (float)(1 + (i - 1) * fs);
}

// Epilogue role of tc_accumulate_kernel (warps 4-7, one per 32-lane tensor-memory quadrant): at
// the end of each accumulator interval add L1 into L2 (or, at the end of a unit, L2 + L1 into the
// FP64 sums) and preload L1 for the next interval.
template <int SK>
__device__ __forceinline__ void epilogue_role(const Params& P, Bars* bars, uint32_t tmem, int warp,
                                              int lane, int fs) {
  const int q = warp & 3;                          // tensor-memory lane quadrant
  const uint32_t lane_addr = tmem + ((uint32_t)(32 * q) << 16);
  uint32_t k = 0;
  bool alive = true;
  for (int64_t u = blockIdx.x; u < P.nunits && alive; u += gridDim.x) {
    const TileInfo ti = decode_tile(P.tiles[u % P.ntiles], P.w != nullptr);
    const int64_t sa = (u / P.ntiles) * P.range_len;
    const int64_t sb = min(P.ns, sa + P.range_len);
    const int nst = (int)((sb - sa + SK - 1) / SK);
    const int nint = interval_count(nst, fs);
    for (int it = 0; it < nint; ++it, ++k) {
      alive = mbar_wait(&bars->l1_full, k & 1, bars, P.err, 13);
      if (!alive) break;
      tc_fence_after();
      const bool first = it == 0, last = it == nint - 1;
      // four K-steps per stage: 64 BF16 samples of K = 16, or 32 TF32 samples of K = 8
      const float c_this = first ? 0.0f : preload_coef(it, nst, fs, 4);
      const float c_next = last ? 0.0f : preload_coef(it + 1, nst, fs, 4);
      const int row = 32 * q + lane;
      const bool vrow = row < ti.nA;
      for (int cc = 0; cc < 256; cc += 32) {
        uint32_t a[32], b[32];
        TMEM_LD32(lane_addr + cc, a);
        if (!first) TMEM_LD32(lane_addr + 256 + cc, b);
        tmem_wait_ld();
        if (last) {
          if (vrow) {
            double* orow = ti.out + (int64_t)(ti.row0 + row) * 2 * ti.m + ti.col0 + cc;
            const int ncol = min(32, ti.nB - cc);
#pragma unroll
            for (int i = 0; i < 32; ++i) {
              if (i < ncol) {
                const float tot = first ? 0.0f : __uint_as_float(b[i]);
                const float d0 = c_this * tot;      // the value this interval started from
                atomicAdd(orow + i, (double)tot + ((double)__uint_as_float(a[i]) - (double)d0));
              }
            }
          }
        } else {
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const float tot = first ? 0.0f : __uint_as_float(b[i]);
            const float d0 = c_this * tot;
            const float nt = tot + (__uint_as_float(a[i]) - d0);
            b[i] = __float_as_uint(nt);
            a[i] = __float_as_uint(c_next * nt);
          }
          TMEM_ST32(lane_addr + 256 + cc, b);
          TMEM_ST32(lane_addr + cc, a);
        }
      }
      tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars->l1_empty);
    }
  }
}

template <bool TF>
__global__ void __launch_bounds__(kThreads, 1) tc_accumulate_kernel(const Params P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  Bars* bars = (Bars*)(smem + kBarOffset);
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&bars->op_full[s], kConvWarps);
      mbar_init(&bars->op_empty[s], 1);
    }
    mbar_init(&bars->l1_full, 1);
    mbar_init(&bars->l1_empty, 4);
    mbar_init(&bars->drain, 1);
    bars->abort = 0;
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
    uint32_t g = 0, k = 0;
    bool alive = true;
    for (int64_t u = blockIdx.x; u < P.nunits && alive; u += gridDim.x) {
      const TileInfo ti = decode_tile(P.tiles[u % P.ntiles], P.w != nullptr);
      const int64_t sa = (u / P.ntiles) * P.range_len;
      const int64_t sb = min(P.ns, sa + P.range_len);
      const int nst = (int)((sb - sa + stage_k<TF>() - 1) / stage_k<TF>());
      for (int st = 0; st < nst && alive; ++st, ++g) {
        const uint32_t slot = g % kStages, use = g / kStages;
        uint32_t acc = 1;
        const bool istart = (st == 0) || ((st - 1) % fs == 0);
        const bool iend = (st == 0) || ((st - 1) % fs == fs - 1) || (st == nst - 1);
        if (istart) {
          // interval 0 starts from zero; later intervals from the epilogue's preloaded value
          alive = mbar_wait(&bars->l1_empty, (k & 1) ^ 1, bars, P.err, 11);
          tc_fence_after();
          acc = (st == 0) ? 0 : 1;
        }
        if (alive) alive = mbar_wait(&bars->op_full[slot], use & 1, bars, P.err, 12);
        if (!alive) break;
        tc_fence_after();
        if (lane == 0) {
          uint8_t* stage = smem + slot * kStageBytes;
          const uint32_t bh = smem_u32(stage), bl = bh + kBBytes;
          uint32_t ah, al;
          if (ti.amode == A_VIEW) {
            ah = bh + (uint32_t)(ti.row0 - ti.pb) * 128u;
            al = bl + (uint32_t)(ti.row0 - ti.pb) * 128u;
          } else {
            ah = bh + 2 * kBBytes;
            al = ah + kABytes;
          }
          // four K-steps of 32 bytes per 128-byte operand row
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const uint32_t o = ks * 32;
            if (TF) {
              mma_tf32(tmem, sdesc(ah + o), sdesc(bh + o), acc);
              mma_tf32(tmem, sdesc(ah + o), sdesc(bl + o), 1);
              mma_tf32(tmem, sdesc(al + o), sdesc(bh + o), 1);
            } else {
              mma_bf16(tmem, sdesc(ah + o), sdesc(bh + o), acc);
              mma_bf16(tmem, sdesc(ah + o), sdesc(bl + o), 1);
              mma_bf16(tmem, sdesc(al + o), sdesc(bh + o), 1);
              mma_bf16(tmem, sdesc(al + o), sdesc(bl + o), 1);
            }
            acc = 1;
          }
          mma_commit(&bars->op_empty[slot]);
          if (iend) mma_commit(&bars->l1_full);
        }
        __syncwarp();
        if (iend) ++k;
      }
    }
    // drain: wait until every issued MMA has completed before tensor memory is released
    if (lane == 0) mma_commit(&bars->drain);
    __syncwarp();
    for (uint32_t i = 0; i < kWaitLimit && !mbar_try_wait(&bars->drain, 0); ++i) {
    }
  } else if (warp >= 4 && warp < 8) {
    epilogue_role<stage_k<TF>()>(P, bars, tmem, warp, lane, fs);
  } else {
    // ------------------------------- converters -------------------------------
    const int cw = warp < 4 ? warp - 1 : warp - 5;   // 0 .. kConvWarps-1
    uint32_t g = 0;
    bool alive = true;
    for (int64_t u = blockIdx.x; u < P.nunits && alive; u += gridDim.x) {
      const TileInfo ti = decode_tile(P.tiles[u % P.ntiles], P.w != nullptr);
      const int64_t sa = (u / P.ntiles) * P.range_len;
      const int64_t sb = min(P.ns, sa + P.range_len);
      const int nst = (int)((sb - sa + stage_k<TF>() - 1) / stage_k<TF>());
      const int halves = TF ? 1 : 2;               // 32-sample halves per stage
      const int njobs_b = (kBRows / 32) * halves;
      // float4 rows need 16-byte aligned parameter offsets and row strides
      const bool vec = P.vec_ok && ((ti.lo + ti.pb) % 4 == 0) && ((ti.lo + ti.row0) % 4 == 0) &&
                       (ti.nB % 4 == 0) && (ti.nA % 4 == 0);
      const int njobs = njobs_b + (ti.amode == A_SEPARATE ? (kARows / 32) * halves : 0);
      for (int st = 0; st < nst; ++st, ++g) {
        const uint32_t slot = g % kStages, use = g / kStages;
        alive = mbar_wait(&bars->op_empty[slot], (use & 1) ^ 1, bars, P.err, 14);
        if (!alive) break;
        uint8_t* stage = smem + slot * kStageBytes;
        const int64_t base = sa + (int64_t)st * stage_k<TF>();
        for (int j = cw; j < njobs; j += kConvWarps) {
          const int kind = j < njobs_b ? 0 : 1;
          const int jj = kind ? j - njobs_b : j;
          const int rg = TF ? jj : jj >> 1, hf = TF ? 0 : (jj & 1);
          if (vec)
            convert_job<true, TF>(P, ti, kind, rg, hf, base, sb, stage);
          else
            convert_job<false, TF>(P, ti, kind, rg, hf, base, sb, stage);
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars->op_full[slot]);
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem)
                 : "memory");
  }
}

// Samples per operand stage of the TMA-fed kernel (two K steps of 16 per 128-byte row half).
constexpr int kTmaStageK = 32;

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
//   HH (columns 0-255)   the hi*hi products, in preloaded intervals of kFlushSamples samples;
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
// The MMA warp issues each stage's corrections before its hi*hi products, so that while the
// epilogue drains HH at an interval boundary the tensor pipe works on CR.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ int stages_through(int i, int nst, int fs) {
  return i == 0 ? 1 : min(nst, 1 + i * fs);
}
// Two K-steps (of 16 samples) per 32-sample stage: an interval of len stages has 2 len levels.
__device__ __forceinline__ float split_kappa(int i, int nst, int fs) {
  const int len = interval_len(i + 1, nst, fs);
  return -centre_frac(2 * len) * (float)len / (float)stages_through(i, nst, fs);
}

__device__ __forceinline__ void epilogue_split_role(const Params& P, Bars* bars, uint32_t tmem,
                                                    int warp, int lane, int fs) {
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
    const TileInfo ti = decode_tile(P.tiles[u % P.ntiles], P.w != nullptr);
    if (row < ti.nA) {
      double* orow = ti.out + (int64_t)(ti.row0 + row) * 2 * ti.m + ti.col0 + 128 * h;
      const int ncol = min(128, ti.nB - 128 * h);
#pragma unroll
      for (int i = 0; i < 128; ++i)
        if (i < ncol) atomicAdd(orow + i, (double)U[i]);
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

__global__ void __maxnreg__(168)
tc_op_kernel(const Params P, const __grid_constant__ CUtensorMap mapA,
             const __grid_constant__ CUtensorMap mapBS, const __grid_constant__ CUtensorMap mapBH) {
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
      const TileInfo ti = decode_tile(P.tiles[u % P.ntiles], P.w != nullptr);
      const int64_t sa = (u / P.ntiles) * P.range_len;
      const int64_t sb = min(P.ns, sa + P.range_len);
      const int nst = (int)((sb - sa + kTmaStageK - 1) / kTmaStageK);
      for (int st = 0; st < nst && alive; ++st, ++g) {
        const uint32_t slot = g % kOpStagesP, use = g / kOpStagesP;
        uint32_t acc = 1;
        const bool istart = (st == 0) || ((st - 1) % fs == 0);
        const bool iend = (st == 0) || ((st - 1) % fs == fs - 1) || (st == nst - 1);
        if (alive && st == 0) {
          // the unit's first correction product overwrites CR: the previous unit's CR must
          // have been read
          alive = mbar_wait(&bars->db_empty[1], (j & 1) ^ 1, bars, P.err, 17);
          tc_fence_after();
        }
        if (alive) alive = mbar_wait(&bars->op_full[slot], use & 1, bars, P.err, 12);
        if (!alive) break;
        tc_fence_after();
        const uint32_t ob = smem_u32(smem + slot * kPStageBytes);
        const uint32_t oa = (ti.amode == A_VIEW) ? ob + (uint32_t)(ti.row0 - ti.pb) * 128u
                                                 : ob + (uint32_t)kBRows * 128u;
        if (lane == 0) {
          // corrections first: they keep the tensor pipe busy while HH is drained
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            const uint32_t o = ks * 32;
            mma_bf16(tmem + 256u, sdesc(oa + o), sdesc(ob + 64 + o),              // hi * lo
                     (st == 0 && ks == 0) ? 0u : 1u);
            mma_bf16(tmem + 256u, sdesc(oa + 64 + o), sdesc(ob + o), 1);        // lo * hi
            mma_bf16(tmem + 256u, sdesc(oa + 64 + o), sdesc(ob + 64 + o), 1);   // lo * lo
          }
        }
        __syncwarp();
        if (istart) {
          // interval 0 of a unit starts HH from zero, later intervals from the epilogue's
          // preload: either way the previous interval's drain must be complete
          alive = mbar_wait(&bars->db_empty[0], (k & 1) ^ 1, bars, P.err, 11);
          tc_fence_after();
          acc = (st == 0) ? 0 : 1;
        }
        if (lane == 0) {
          if (alive) {
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
              mma_bf16(tmem, sdesc(oa + ks * 32), sdesc(ob + ks * 32), acc);   // hi * hi
              acc = 1;
            }
          }
          mma_commit(&bars->op_empty[slot]);
          if (alive && iend) mma_commit(&bars->db_full[0]);
          if (alive && st == nst - 1) mma_commit(&bars->db_full[1]);
        }
        __syncwarp();
        if (iend) ++k;
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
      const TileInfo ti = decode_tile(P.tiles[u % P.ntiles], P.w != nullptr);
      const int64_t sa = (u / P.ntiles) * P.range_len;
      const int64_t sb = min(P.ns, sa + P.range_len);
      const int nst = (int)((sb - sa + kTmaStageK - 1) / kTmaStageK);
      const bool aview = ti.amode == A_VIEW;
      const uint32_t bytes = (uint32_t)kBRows * 128u + (aview ? 0u : (uint32_t)kARows * 128u);
      const CUtensorMap* mb = ti.xtype ? &mapBH : &mapBS;
      for (int st = 0; st < nst && alive; ++st, ++g) {
        const uint32_t slot = g % kOpStagesP, use = g / kOpStagesP;
        alive = mbar_wait(&bars->op_empty[slot], (use & 1) ^ 1, bars, P.err, 15);
        if (!alive) break;
        if (lane == 0) {
          uint64_t* bar = &bars->op_full[slot];
          const uint32_t dst = smem_u32(smem + slot * kPStageBytes);
          const int x = (int)((sa / kTmaStageK + st) * 64);
          mbar_expect_tx(bar, bytes);
          tma_load_2d(dst, mb, x, (int)(ti.lo + ti.pb), bar);
          if (!aview) tma_load_2d(dst + kBRows * 128, &mapA, x, (int)(ti.lo + ti.row0), bar);
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
    epilogue_split_role(P, bars, tmem, warp, lane, fs);
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

bool tc_supported() { return true; }

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

cudaError_t launch_tc_accumulate(const float* Y, const float* Z, const float* E, const float* w,
                                 int64_t ns, int64_t ncols, int64_t ld, const float* shift32,
                                 const TcTile* tiles, int ntiles, int32_t* err, int tf32,
                                 cudaStream_t st) {
  if (ns <= 0 || ntiles <= 0) return cudaSuccess;
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(tc_accumulate_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kSmemBytes);
    cudaFuncSetAttribute(tc_accumulate_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kSmemBytes);
  }
  Params P;
  P.Y = Y;
  P.Z = Z;
  P.E = E;
  P.w = w;
  P.shift = shift32;
  P.ns = ns;
  P.ld = ld;
  P.tiles = tiles;
  P.ntiles = ntiles;
  // sample ranges: enough units to keep every SM busy with a small tail, but never shorter
  // than kMinUnitSamples, so that the preloaded intervals (not the unpreloaded first stage)
  // carry nearly all of every unit's sum
  int64_t range = 8192;
  const int64_t sk = tf32 ? kStageKTf : kStageK;
  while (range > kMinUnitSamples && ((ns + range - 1) / range) * ntiles < 8LL * sms) range /= 2;
  P.range_len = range;
  P.nunits = ((ns + range - 1) / range) * ntiles;
  P.flush_stages = (int)(kFlushSamples / sk) > 0 ? (int)(kFlushSamples / sk) : 1;
  P.err = err;
  P.vec_ok = (ld % 4 == 0) && (((uintptr_t)Y | (uintptr_t)Z) % 16 == 0);
  const int grid = (int)(P.nunits < sms ? P.nunits : sms);
  if (tf32)
    tc_accumulate_kernel<true><<<grid, kThreads, kSmemBytes, st>>>(P);
  else
    tc_accumulate_kernel<false><<<grid, kThreads, kSmemBytes, st>>>(P);
  return cudaGetLastError();
}


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

cudaError_t launch_tc_prepared(const uint8_t* opA, const uint8_t* opBS, const uint8_t* opBH,
                               int64_t nrows, int64_t row_bytes, int64_t ns, const TcTile* tiles,
                               int ntiles, int weighted, int32_t* err, cudaStream_t st) {
  if (ns <= 0 || ntiles <= 0) return cudaSuccess;
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(tc_op_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kPSmemBytes);
  }
  CUtensorMap mA, mBS, mBH;
  if (!encode_op_map(&mA, opA, nrows, row_bytes, kARows) ||
      !encode_op_map(&mBS, weighted ? opBS : opA, nrows, row_bytes, kBRows) ||
      !encode_op_map(&mBH, opBH, nrows, row_bytes, kBRows))
    return cudaErrorInvalidValue;
  Params P;
  P.Y = nullptr;
  P.Z = nullptr;
  P.E = nullptr;
  // decode_tile takes A as a view of B only without weights; the pointer is not dereferenced
  P.w = weighted ? reinterpret_cast<const float*>(opBS) : nullptr;
  P.shift = nullptr;
  P.ns = ns;
  P.ld = 0;
  P.tiles = tiles;
  P.ntiles = ntiles;
  // sample ranges of up to 16384 (512 stages): each unit ends in one flush of its sums with
  // FP64 atomics and one wait for its first interval's drain, so units are kept long; at
  // least four units per SM keep the tail short
  int64_t range = 16384;
  while (range > kMinUnitSamples && ((ns + range - 1) / range) * ntiles < 4LL * sms) range /= 2;
  P.range_len = range;
  P.nunits = ((ns + range - 1) / range) * ntiles;
  P.flush_stages = kFlushSamples / kTmaStageK;
  P.err = err;
  P.vec_ok = 0;
  const int grid = (int)(P.nunits < sms ? P.nunits : sms);
  tc_op_kernel<<<grid, kPThreads, kPSmemBytes, st>>>(P, mA, mBS, mBH);
  return cudaGetLastError();
}

}  // namespace blm
