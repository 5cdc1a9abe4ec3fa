// Operand preparation for the split-precision sweeps (Eq. 3 / Eq. 5 / Eq. 7 sums on tensor
// cores), fused with the first-moment sums of the same sweep.
//
// Each FP32 sample element is converted once per sweep into the operands of the tensor-core
// contraction, stored in HBM in the layout the tensor core reads (K-major, one 128-byte row per
// parameter and sample group: [hi(32 samples) | lo(32 samples)] in bf16, or [hi(16) | lo(16)]
// in TF32):
//   opA  = Y' = Y - c                       (A operand, all tiles)
//   opBH = w (E Y' + Z)                     (B operand of the Hamiltonian tiles, X')
//   opBS = w Y'                             (B operand of the overlap tiles when weighted;
//                                            without weights those tiles read opA)
// so that the contraction kernel is TMA + MMA only.  The same pass accumulates the first moments
// sum w Y', sum w E Y', sum w Z per parameter (and sum w, sum w E) into FP64, in FP32 runs of 64
// samples per thread and parameter.
//
// A CTA takes 64 parameters x 1024 samples in tiles of 64 samples; thread (p4, sb) owns
// parameters 4 p4 .. 4 p4 + 3 and samples 8 sb .. 8 sb + 7 of a tile and writes one 16-byte
// store per parameter for hi and one for lo.  prep_direct_kernel (16-byte aligned rows, the
// usual case) loads its tile straight into registers; prep_kernel (any alignment) stages it
// through shared memory with cp.async, double-buffered.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "blm_internal.cuh"

namespace blm {

namespace {

constexpr int kPrepP = 64;             // parameters per CTA
constexpr int kPrepT = 64;             // samples per tile (two 32-sample groups)
constexpr int kPrepTiles = 16;         // tiles per CTA
constexpr int kPrepThreads = 128;      // 16 parameter quads x 8 sample blocks
constexpr int kPrepLd = kPrepP + 4;    // padded row (16-byte aligned)
constexpr int kPrepRun = 8;            // tiles per FP32 run of the sums (64 samples per thread)
constexpr int kPrepBufFloats = 2 * kPrepT * kPrepLd + 2 * kPrepT;   // O, G, E, W of one tile
constexpr size_t kPrepSmem = 2 * kPrepBufFloats * sizeof(float);

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

// hi/lo split of 4 values for the TF32 products: hi = v rounded to 8 significant bits (a bf16
// value, exact in TF32), lo = tf32(v - hi) (11 bits, round to nearest); both have their low 13
// bits zero, so the tensor core reads them exactly, and hi + lo represents v to 2^-21.  hi keeps
// as few bits as the BF16 split's so that the hi*hi products (16 significant bits) lose as
// little to the accumulator's truncation as there.
__device__ __forceinline__ void split4_tf32(const float* v, uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t hb = pack_bf16x2(v[k], 0.0f);          // bf16(v) in the low half
    h[k] = hb << 16;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l[k]) : "f"(v[k] - __uint_as_float(h[k])));
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Writes one thread's 8 consecutive samples (tile-relative sample 8 sb, tile start s0t) of one
// parameter row: BF16 rows hold 32-sample groups [hi(32) | lo(32)] of 2 bytes, TF32 rows
// 16-sample groups [hi(16) | lo(16)] of 4 bytes; both are 128 bytes per group.
template <bool TF>
__device__ __forceinline__ void store_split8(uint8_t* row, int64_t s0t, int sb, const float* v) {
  if (TF) {
    const int64_t grp = s0t / 16 + (sb >> 1);
    uint8_t* base = row + grp * 128 + 32 * (sb & 1);
    uint4 hi, lo;
    split4_tf32(v, hi, lo);
    *reinterpret_cast<uint4*>(base) = hi;
    *reinterpret_cast<uint4*>(base + 64) = lo;
    split4_tf32(v + 4, hi, lo);
    *reinterpret_cast<uint4*>(base + 16) = hi;
    *reinterpret_cast<uint4*>(base + 80) = lo;
  } else {
    const int64_t grp = s0t / 32 + (sb >> 2);
    uint8_t* base = row + grp * 128 + 16 * (sb & 3);
    uint4 hi, lo;
    split8_bf16(v, hi, lo);
    *reinterpret_cast<uint4*>(base) = hi;
    *reinterpret_cast<uint4*>(base + 64) = lo;
  }
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

struct PrepArgs {
  const float* Y;
  const float* Z;
  const float* E;
  const float* w;
  int64_t ns, ld, n;
  const float* shift;     // per-parameter c, or nullptr
  uint8_t* opA;
  uint8_t* opBS;          // nullptr without weights
  uint8_t* opBH;
  int64_t row_bytes;
  double* sY;             // first moments (FP64 sums), or nullptr
  double* sEY;
  double* sZ;
  double* scal;           // sum w, sum w E (CTAs of the first parameter tile), or nullptr
  int vec;                // 16-byte copies allowed
};

template <bool TF>
__global__ void __launch_bounds__(kPrepThreads)
prep_kernel(const PrepArgs a) {
  extern __shared__ __align__(16) float sm[];
  const int t = threadIdx.x;
  const int p4 = t & 15, sb = t >> 4;
  const int64_t p0 = (int64_t)blockIdx.x * kPrepP;
  const int64_t sbase = (int64_t)blockIdx.y * kPrepT * kPrepTiles;
  const int ntiles = (int)min((int64_t)kPrepTiles, (a.ns - sbase + kPrepT - 1) / kPrepT);

  auto issue = [&](int ti) {
    float* buf = sm + (ti & 1) * kPrepBufFloats;
    float* Os = buf;
    float* Gs = Os + kPrepT * kPrepLd;
    float* Es = Gs + kPrepT * kPrepLd;
    const int64_t s0 = sbase + (int64_t)ti * kPrepT;
    if (a.vec) {
#pragma unroll
      for (int i = 0; i < kPrepT * kPrepP / 4 / kPrepThreads; ++i) {
        const int idx = t + i * kPrepThreads;
        const int s = idx >> 4, q = idx & 15;
        const int64_t p = p0 + 4 * q;
        const bool srow = s0 + s < a.ns;
        const int valid = (int)(srow ? max((int64_t)0, min((int64_t)4, a.n - p)) : 0);
        const int64_t off = valid ? (s0 + s) * a.ld + p : 0;
        cp_async16(Os + s * kPrepLd + 4 * q, a.Y + off, 4 * valid);
        cp_async16(Gs + s * kPrepLd + 4 * q, a.Z + off, 4 * valid);
      }
    } else {
#pragma unroll 8
      for (int i = 0; i < kPrepT * kPrepP / kPrepThreads; ++i) {
        const int idx = t + i * kPrepThreads;
        const int s = idx / kPrepP, p = idx % kPrepP;
        const bool ok = (s0 + s < a.ns) && (p0 + p < a.n);
        const int64_t off = ok ? (s0 + s) * a.ld + p0 + p : 0;
        cp_async4(Os + s * kPrepLd + p, a.Y + off, ok);
        cp_async4(Gs + s * kPrepLd + p, a.Z + off, ok);
      }
    }
    if (t < kPrepT) {
      const bool ok = s0 + t < a.ns;
      cp_async4(Es + t, a.E + (ok ? s0 + t : 0), ok);
      if (a.w) cp_async4(Es + kPrepT + t, a.w + (ok ? s0 + t : 0), ok);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };

  float c[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int64_t p = p0 + 4 * p4 + e;
    c[e] = (a.shift && p < a.n) ? __ldg(a.shift + p) : 0.0f;
  }
  double dY[4] = {0, 0, 0, 0}, dEY[4] = {0, 0, 0, 0}, dZ[4] = {0, 0, 0, 0};
  float fY[4] = {0, 0, 0, 0}, fEY[4] = {0, 0, 0, 0}, fZ[4] = {0, 0, 0, 0};
  double dW = 0.0, dWE = 0.0;
  const bool scal_thread = a.scal && blockIdx.x == 0 && p4 == 0;

  issue(0);
  for (int ti = 0; ti < ntiles; ++ti) {
    if (ti + 1 < ntiles) {
      issue(ti + 1);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    const float* buf = sm + (ti & 1) * kPrepBufFloats;
    const float* Os = buf;
    const float* Gs = Os + kPrepT * kPrepLd;
    const float* Es = Gs + kPrepT * kPrepLd;
    const int64_t s0 = sbase + (int64_t)ti * kPrepT;
    float ya[4][8], xb[4][8], yb[4][8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int s = 8 * sb + j;
      const bool ok = s0 + s < a.ns;
      const float4 o = *reinterpret_cast<const float4*>(Os + s * kPrepLd + 4 * p4);
      const float4 g = *reinterpret_cast<const float4*>(Gs + s * kPrepLd + 4 * p4);
      const float ev = Es[s];
      const float wv = ok ? (a.w ? Es[kPrepT + s] : 1.0f) : 0.0f;
      if (scal_thread && sb >= 0) {
        dW += (double)wv;
        dWE += (double)(wv * ev);
      }
      const float ov[4] = {o.x, o.y, o.z, o.w}, gv[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float y = ok ? ov[e] - c[e] : 0.0f;
        const float wy = wv * y;
        ya[e][j] = y;
        yb[e][j] = wy;
        xb[e][j] = wv * fmaf(ev, y, gv[e]);
        fY[e] += wy;
        fEY[e] = fmaf(wy, ev, fEY[e]);
        fZ[e] = fmaf(wv, gv[e], fZ[e]);
      }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int64_t p = p0 + 4 * p4 + e;
      if (p >= a.n) continue;
      store_split8<TF>(a.opA + p * a.row_bytes, s0, sb, ya[e]);
      store_split8<TF>(a.opBH + p * a.row_bytes, s0, sb, xb[e]);
      if (a.opBS) store_split8<TF>(a.opBS + p * a.row_bytes, s0, sb, yb[e]);
    }
    if ((ti + 1) % kPrepRun == 0 || ti + 1 == ntiles) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        dY[e] += (double)fY[e];
        dEY[e] += (double)fEY[e];
        dZ[e] += (double)fZ[e];
        fY[e] = fEY[e] = fZ[e] = 0.0f;
      }
    }
    __syncthreads();
  }
  if (a.sY) {
    // the 8 sample blocks of a parameter quad: lanes p4 and p4 + 16 of a warp, then the 4 warps
    double* red = reinterpret_cast<double*>(sm);   // tile buffers are free now
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      dY[e] += __shfl_xor_sync(0xffffffffu, dY[e], 16);
      dEY[e] += __shfl_xor_sync(0xffffffffu, dEY[e], 16);
      dZ[e] += __shfl_xor_sync(0xffffffffu, dZ[e], 16);
    }
    const int wid = t >> 5, lane = t & 31;
    if (lane < 16) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        red[((wid * 16 + lane) * 4 + e) * 3 + 0] = dY[e];
        red[((wid * 16 + lane) * 4 + e) * 3 + 1] = dEY[e];
        red[((wid * 16 + lane) * 4 + e) * 3 + 2] = dZ[e];
      }
    }
    __syncthreads();
    if (t < kPrepP) {
      const int q = t >> 2, e = t & 3;
      const int64_t p = p0 + t;
      double s1 = 0.0, s2 = 0.0, s3 = 0.0;
      for (int w4 = 0; w4 < kPrepThreads / 32; ++w4) {
        s1 += red[((w4 * 16 + q) * 4 + e) * 3 + 0];
        s2 += red[((w4 * 16 + q) * 4 + e) * 3 + 1];
        s3 += red[((w4 * 16 + q) * 4 + e) * 3 + 2];
      }
      if (p < a.n) {
        atomicAdd(a.sY + p, s1);
        atomicAdd(a.sEY + p, s2);
        atomicAdd(a.sZ + p, s3);
      }
    }
  }
  if (scal_thread) {
    atomicAdd(a.scal + 0, dW);
    atomicAdd(a.scal + 1, dWE);
  }
}

// ---------------------------------------------------------------------------------------------
// The same preparation with the tiles read straight into registers (16-byte rows aligned):
// no shared-memory staging and no barriers in the loop, so occupancy is set by registers alone
// (four CTAs of 128 threads per SM instead of three) and each thread keeps its tile's sixteen
// 16-byte loads in flight.  The FP64 partial sums live in a per-thread shared-memory slot.
// ---------------------------------------------------------------------------------------------
constexpr int kPdThreads = 128;

template <bool WT, bool TF>
__global__ void __launch_bounds__(kPdThreads, 4)
prep_direct_kernel(const PrepArgs a) {
  __shared__ double dsum[kPdThreads * 12];   // per thread: sY[4], sEY[4], sZ[4]; then reduction
  const int t = threadIdx.x;
  const int p4 = t & 15, sb = t >> 4;
  const int64_t p0 = (int64_t)blockIdx.x * kPrepP;
  const int64_t pq = p0 + 4 * p4;                      // this thread's first parameter
  const int64_t sbase = (int64_t)blockIdx.y * kPrepT * kPrepTiles;
  const int ntiles = (int)min((int64_t)kPrepTiles, (a.ns - sbase + kPrepT - 1) / kPrepT);
  const int nval = (int)max((int64_t)0, min((int64_t)4, a.n - pq));   // valid parameters
  float c[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) c[e] = (a.shift && e < nval) ? __ldg(a.shift + pq + e) : 0.0f;
  double* my = dsum + t * 12;
#pragma unroll
  for (int i = 0; i < 12; ++i) my[i] = 0.0;
  float fY[4] = {0, 0, 0, 0}, fEY[4] = {0, 0, 0, 0}, fZ[4] = {0, 0, 0, 0};
  double dW = 0.0, dWE = 0.0;
  const bool scal_thread = a.scal && blockIdx.x == 0 && p4 == 0;

  for (int ti = 0; ti < ntiles; ++ti) {
    const int64_t s0 = sbase + (int64_t)ti * kPrepT + 8 * sb;   // this thread's 8 samples
    float4 o[8], g[8];
    float ev[8], wv[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int64_t s = s0 + j;
      const bool ok = s < a.ns;
      o[j] = g[j] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if (ok && nval == 4) {
        o[j] = __ldcs(reinterpret_cast<const float4*>(a.Y + s * a.ld + pq));
        g[j] = __ldcs(reinterpret_cast<const float4*>(a.Z + s * a.ld + pq));
      } else if (ok) {   // the last, partial quad of parameters
        const float* yr = a.Y + s * a.ld + pq;
        const float* zr = a.Z + s * a.ld + pq;
        o[j] = make_float4(nval > 0 ? yr[0] : 0.0f, nval > 1 ? yr[1] : 0.0f, nval > 2 ? yr[2] : 0.0f, 0.0f);
        g[j] = make_float4(nval > 0 ? zr[0] : 0.0f, nval > 1 ? zr[1] : 0.0f, nval > 2 ? zr[2] : 0.0f, 0.0f);
      }
      ev[j] = ok ? __ldg(a.E + s) : 0.0f;
      wv[j] = ok ? (WT ? __ldg(a.w + s) : 1.0f) : 0.0f;
    }
    float ya[4][8], xb[4][8], yb[WT ? 4 : 1][8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (scal_thread) {
        dW += (double)wv[j];
        dWE += (double)(wv[j] * ev[j]);
      }
      const float ov[4] = {o[j].x, o[j].y, o[j].z, o[j].w}, gv[4] = {g[j].x, g[j].y, g[j].z, g[j].w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float y = (s0 + j < a.ns) ? ov[e] - c[e] : 0.0f;
        const float wy = wv[j] * y;
        ya[e][j] = y;
        if (WT) yb[WT ? e : 0][j] = wy;
        xb[e][j] = wv[j] * fmaf(ev[j], y, gv[e]);
        fY[e] += wy;
        fEY[e] = fmaf(wy, ev[j], fEY[e]);
        fZ[e] = fmaf(wv[j], gv[e], fZ[e]);
      }
    }
    const int64_t s0t = sbase + (int64_t)ti * kPrepT;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (e >= nval) continue;
      store_split8<TF>(a.opA + (pq + e) * a.row_bytes, s0t, sb, ya[e]);
      store_split8<TF>(a.opBH + (pq + e) * a.row_bytes, s0t, sb, xb[e]);
      if (WT) store_split8<TF>(a.opBS + (pq + e) * a.row_bytes, s0t, sb, yb[WT ? e : 0]);
    }
    if ((ti + 1) % kPrepRun == 0 || ti + 1 == ntiles) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        my[e] += (double)fY[e];
        my[4 + e] += (double)fEY[e];
        my[8 + e] += (double)fZ[e];
        fY[e] = fEY[e] = fZ[e] = 0.0f;
      }
    }
  }
  if (a.sY) {
    // the 8 sample blocks of a parameter quad: threads p4 + 16 sb, sb = 0..7
    __syncthreads();
    if (t < kPrepP) {
      const int q = t >> 2, e = t & 3;
      double s1 = 0.0, s2 = 0.0, s3 = 0.0;
      for (int b8 = 0; b8 < 8; ++b8) {
        const double* src = dsum + (q + 16 * b8) * 12;
        s1 += src[e];
        s2 += src[4 + e];
        s3 += src[8 + e];
      }
      const int64_t p = p0 + t;
      if (p < a.n) {
        atomicAdd(a.sY + p, s1);
        atomicAdd(a.sEY + p, s2);
        atomicAdd(a.sZ + p, s3);
      }
    }
  }
  if (scal_thread) {
    atomicAdd(a.scal + 0, dW);
    atomicAdd(a.scal + 1, dWE);
  }
}

}  // namespace

void launch_prep(const float* Y, const float* Z, const float* E, const float* w, int64_t ns,
                 int64_t ld, int64_t n, const float* shift32, uint8_t* opA, uint8_t* opBS,
                 uint8_t* opBH, int64_t row_bytes, double* sY, double* sEY, double* sZ,
                 double* scal, int tf32, cudaStream_t st) {
  if (ns <= 0) return;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(prep_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPrepSmem);
    cudaFuncSetAttribute(prep_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPrepSmem);
    attr = true;
  }
  PrepArgs a{Y, Z, E, w, ns, ld, n, shift32, opA, w ? opBS : nullptr, opBH, row_bytes,
             sY, sEY, sZ, scal,
             (ld % 4 == 0) && ((((uintptr_t)Y) | ((uintptr_t)Z)) % 16 == 0) ? 1 : 0};
  dim3 grid((unsigned)((n + kPrepP - 1) / kPrepP),
            (unsigned)((ns + kPrepT * kPrepTiles - 1) / (kPrepT * kPrepTiles)));
  if (tf32) {
    if (a.vec && w)
      prep_direct_kernel<true, true><<<grid, kPdThreads, 0, st>>>(a);
    else if (a.vec)
      prep_direct_kernel<false, true><<<grid, kPdThreads, 0, st>>>(a);
    else
      prep_kernel<true><<<grid, kPrepThreads, kPrepSmem, st>>>(a);
  } else {
    if (a.vec && w)
      prep_direct_kernel<true, false><<<grid, kPdThreads, 0, st>>>(a);
    else if (a.vec)
      prep_direct_kernel<false, false><<<grid, kPdThreads, 0, st>>>(a);
    else
      prep_kernel<false><<<grid, kPrepThreads, kPrepSmem, st>>>(a);
  }
}

}  // namespace blm
