// Operand preparation for the split-BF16 first sweep (Eq. 3 / Eq. 5 sums on tensor cores).
//
// Each FP32 sample element is converted once per sweep into the operands of the tensor-core
// contraction, stored in HBM in the layout the tensor core reads (K-major, one 128-byte row per
// parameter and 32-sample group: [hi(32 samples) | lo(32 samples)] in bf16):
//   opA  = Y' = O - c                       (A operand, all tiles)
//   opBH = w (E Y' + G)                     (B operand of the Hamiltonian tiles, X')
//   opBS = w Y'                             (B operand of the overlap tiles when weighted;
//                                            without weights those tiles read opA)
// so that the contraction kernel is TMA + MMA only.  A CTA takes 64 parameters x 64 samples:
// coalesced FP32 loads of the sample rows into shared memory, then one thread per (parameter,
// 32-sample group) reads its column, splits and writes its three 128-byte rows.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "blm_internal.cuh"

namespace blm {

namespace {

constexpr int kPrepP = 64;            // parameters per CTA
constexpr int kPrepS = 64;            // samples per CTA (2 groups of 32)
constexpr int kPrepThreads = 128;     // one thread per (parameter, group)
constexpr int kPrepLd = kPrepP + 4;   // padded smem row (16-byte aligned): a warp's
                                      // column reads (32 parameters) hit different banks

__device__ __forceinline__ uint32_t pack_bf16x2(float first, float second) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(second), "f"(first));
  return d;
}

// hi/lo split of 8 values: hi = bf16(v), lo = bf16(v - hi)
__device__ __forceinline__ void split8_bf16(const float* v, uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t hh = pack_bf16x2(v[2 * k], v[2 * k + 1]);
    h[k] = hh;
    l[k] = pack_bf16x2(v[2 * k] - __uint_as_float(hh << 16),
                       v[2 * k + 1] - __uint_as_float(hh & 0xFFFF0000u));
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool ok) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(
                   (unsigned)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(ok ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async16(float* dst, const float* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                   (unsigned)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(bytes)
               : "memory");
}

__global__ void __launch_bounds__(kPrepThreads)
prep_kernel(const float* __restrict__ O, const float* __restrict__ G,
            const float* __restrict__ E, const float* __restrict__ w, int64_t ns, int64_t ld,
            int64_t n, const float* __restrict__ shift, uint8_t* __restrict__ opA,
            uint8_t* __restrict__ opBS, uint8_t* __restrict__ opBH, int64_t row_bytes) {
  __shared__ __align__(16) float Os[kPrepS * kPrepLd];
  __shared__ __align__(16) float Gs[kPrepS * kPrepLd];
  __shared__ float Es[kPrepS], Ws[kPrepS];
  const int t = threadIdx.x;
  const int64_t p0 = (int64_t)blockIdx.x * kPrepP;
  const int64_t s0 = (int64_t)blockIdx.y * kPrepS;
  // the whole tile in flight at once (cp.async, zero-filled outside the sample and parameter
  // ranges): 16-byte copies when rows and the tile start are 16-byte aligned
  const bool vec = (ld % 4 == 0) && ((((uintptr_t)O) | ((uintptr_t)G)) % 16 == 0);
  if (vec) {
#pragma unroll
    for (int i = 0; i < kPrepS * kPrepP / 4 / kPrepThreads; ++i) {
      const int idx = t + i * kPrepThreads;          // float4 index in the tile
      const int s = idx / (kPrepP / 4), q = idx % (kPrepP / 4);
      const int64_t p = p0 + 4 * q;
      const bool srow = s0 + s < ns;
      const int valid = (int)(srow ? max((int64_t)0, min((int64_t)4, n - p)) : 0);
      const int64_t off = srow && valid ? (s0 + s) * ld + p : 0;
      cp_async16(Os + s * kPrepLd + 4 * q, O + off, 4 * valid);
      cp_async16(Gs + s * kPrepLd + 4 * q, G + off, 4 * valid);
    }
  } else {
#pragma unroll 8
    for (int i = 0; i < kPrepS * kPrepP / kPrepThreads; ++i) {
      const int idx = t + i * kPrepThreads;
      const int s = idx / kPrepP, p = idx % kPrepP;
      const bool ok = (s0 + s < ns) && (p0 + p < n);
      const int64_t off = ok ? (s0 + s) * ld + p0 + p : 0;
      cp_async4(Os + s * kPrepLd + p, O + off, ok);
      cp_async4(Gs + s * kPrepLd + p, G + off, ok);
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  if (t < kPrepS) {
    const bool ok = s0 + t < ns;
    Es[t] = ok ? __ldg(E + s0 + t) : 0.0f;
    Ws[t] = (ok && w) ? __ldg(w + s0 + t) : (ok ? 1.0f : 0.0f);
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  const int p = t % kPrepP, gq = t / kPrepP;     // parameter, 32-sample group
  const int64_t pg = p0 + p;
  if (pg >= n) return;
  const float c = shift ? __ldg(shift + pg) : 0.0f;
  const int64_t grp = s0 / 32 + gq;              // sample group within the chunk
  const int64_t rowoff = pg * row_bytes + grp * 128;
#pragma unroll
  for (int jb = 0; jb < 4; ++jb) {
    float ya[8], xb[8], yb[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int s = 32 * gq + 8 * jb + j;
      const bool ok = s0 + s < ns;
      const float y = ok ? Os[s * kPrepLd + p] - c : 0.0f;
      const float wv = Ws[s];
      ya[j] = y;
      xb[j] = wv * fmaf(Es[s], y, Gs[s * kPrepLd + p]);
      yb[j] = wv * y;
    }
    uint4 hi, lo;
    split8_bf16(ya, hi, lo);
    *reinterpret_cast<uint4*>(opA + rowoff + 16 * jb) = hi;
    *reinterpret_cast<uint4*>(opA + rowoff + 64 + 16 * jb) = lo;
    split8_bf16(xb, hi, lo);
    *reinterpret_cast<uint4*>(opBH + rowoff + 16 * jb) = hi;
    *reinterpret_cast<uint4*>(opBH + rowoff + 64 + 16 * jb) = lo;
    if (opBS) {
      split8_bf16(yb, hi, lo);
      *reinterpret_cast<uint4*>(opBS + rowoff + 16 * jb) = hi;
      *reinterpret_cast<uint4*>(opBS + rowoff + 64 + 16 * jb) = lo;
    }
  }
}

}  // namespace

void launch_prep(const float* O, const float* G, const float* E, const float* w, int64_t ns,
                 int64_t ld, int64_t n, const float* shift32, uint8_t* opA, uint8_t* opBS,
                 uint8_t* opBH, int64_t row_bytes, cudaStream_t st) {
  if (ns <= 0) return;
  dim3 grid((unsigned)((n + kPrepP - 1) / kPrepP), (unsigned)((ns + kPrepS - 1) / kPrepS));
  prep_kernel<<<grid, kPrepThreads, 0, st>>>(O, G, E, w, ns, ld, n, shift32, opA,
                                             w ? opBS : nullptr, opBH, row_bytes);
}

}  // namespace blm
