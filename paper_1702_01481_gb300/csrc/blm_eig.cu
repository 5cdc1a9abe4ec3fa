// FP64 generalized eigen-solver for the block problems (Eq. 5 / Eq. 10) and the combined problem
// (Eq. 7) of the blocked linear method: H v = lambda S v with H non-symmetric and S symmetric
// positive definite, keeping the eigenpairs with the lowest real parts (Sec. II.B).
//
// One CTA per problem (all blocks in one launch).  Steps, all FP64:
//   1. diagonal scaling  S~ = D S D, H~ = D H D with D = diag(S)^-1/2;
//   2. Cholesky  S~ = L L^T  and reduction to standard form  A = L^-1 H~ L^-T;
//   3. Householder reduction of A to upper Hessenberg form  A = Q Hs Q^T;
//   4. Francis double-shift QR on Hs for all eigenvalues (eigenvalues only, active window),
//      the bulge chased through shared-memory windows (hqr_windowed);
//   5. for each wanted eigenvalue, inverse iteration on the Hessenberg matrix, one warp per
//      eigenvalue (real or complex LU with the one-row partial pivoting a Hessenberg matrix
//      needs), residual-checked;
//   6. back-transformation  v = D L^-T Q y, one warp per direction.
// On this GPU an FP64 operation has ~65 cycles of latency and the SM retires one FP64 warp
// instruction per ~19 cycles, so the QR sweep (a serial chain of reflectors) is latency bound:
// the reflector avoids the FP64 divide and square root (see rcp_nr / rsqrt_nr).
// Iterations are bounded: a QR that does not converge within 40 m sweeps reports ST_NOCONV.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <algorithm>
#include <memory>
#include <vector>

#include "blm_internal.cuh"

namespace blm {

namespace {

constexpr int kEigThreads = 512;
constexpr int kMaxKeep = 64;

struct cplx {
  double re, im;
};
__device__ __forceinline__ cplx cmk(double r, double i) { return cplx{r, i}; }
__device__ __forceinline__ cplx operator-(cplx a, cplx b) { return cmk(a.re - b.re, a.im - b.im); }
__device__ __forceinline__ cplx operator*(cplx a, cplx b) {
  return cmk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
__device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
  // Smith's algorithm
  if (fabs(b.re) >= fabs(b.im)) {
    const double r = b.im / b.re, d = b.re + b.im * r;
    return cmk((a.re + a.im * r) / d, (a.im - a.re * r) / d);
  }
  const double r = b.re / b.im, d = b.re * r + b.im;
  return cmk((a.re * r + a.im) / d, (a.im * r - a.re) / d);
}
__device__ __forceinline__ double cabs2(cplx a) { return fabs(a.re) + fabs(a.im); }


__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  const int nw = blockDim.x >> 5;
  for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}

__device__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  const int nw = blockDim.x >> 5;
  for (int i = 0; i < nw; ++i) s = fmax(s, red[i]);
  return s;
}

// 1/a and 1/sqrt(a) to FP64 accuracy without the FP64 divide and square-root sequences, whose
// latency (about 650 cycles each on this GPU) sits on the QR sweep's critical path: an FP32 seed
// refined by two Newton-Raphson steps, r <- r + r (1 - a r) and r <- r + (r / 2) (1 - a r^2),
// each of which doubles the number of correct bits.  Arguments outside the FP32 range take the
// plain FP64 operation.
__device__ __forceinline__ double rcp_nr(double a) {
  const double aa = fabs(a);
  if (!(aa > 1e-30 && aa < 1e30)) return 1.0 / a;
  double r = (double)__frcp_rn((float)a);
  r = fma(r, fma(-a, r, 1.0), r);
  r = fma(r, fma(-a, r, 1.0), r);
  return r;
}
__device__ __forceinline__ double rsqrt_nr(double a) {
  if (!(a > 1e-30 && a < 1e30)) return 1.0 / sqrt(a);
  double r = (double)rsqrtf((float)a);
  for (int it = 0; it < 2; ++it) {
    const double e = fma(-a * r, r, 1.0);
    r = fma(0.5 * r, e, r);
  }
  return r;
}

// ---------------------------------------------------------------------------------------------
// Double-word arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi) / 2, about 48 significant bits.  On this GPU an FP32 operation has ~4.6 cycles
// of latency against FP64's 65, and the SM's FP32 throughput is ~64x its FP64 throughput, so the
// latency-bound QR sweep runs on double words.  The operations are the error-free transforms
// TwoSum (Knuth), Fast2Sum (Dekker) and the FMA-based exact product, combined as in the
// double-word addition and multiplication algorithms of Joldes, Muller and Popescu (ACM TOMS 44,
// 2017): relative error of an addition <= 3u^2, of a multiplication <= 5u^2, u = 2^-24.
// Explicit _rn intrinsics keep the compiler from contracting or reassociating them.
// ---------------------------------------------------------------------------------------------
struct dw {
  float hi, lo;
};
__device__ __forceinline__ dw dw_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dw{s, e};
}
__device__ __forceinline__ dw dw_fast_two_sum(float a, float b) {   // |a| >= |b| or a = 0
  const float s = __fadd_rn(a, b);
  return dw{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dw operator+(dw x, dw y) {
  const dw s = dw_two_sum(x.hi, y.hi);
  const dw t = dw_two_sum(x.lo, y.lo);
  dw u = dw_fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return dw_fast_two_sum(u.hi, __fadd_rn(u.lo, t.lo));
}
__device__ __forceinline__ dw operator-(dw x) { return dw{-x.hi, -x.lo}; }
__device__ __forceinline__ dw operator-(dw x, dw y) { return x + (-y); }
__device__ __forceinline__ dw operator*(dw x, dw y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, e));
  return dw_fast_two_sum(p, e);
}
__device__ __forceinline__ dw dw_of(float a) { return dw{a, 0.0f}; }
__device__ __forceinline__ dw dw_of_double(double d) {
  const float h = __double2float_rn(d);
  return dw{h, __double2float_rn(d - (double)h)};
}
__device__ __forceinline__ double to_double(dw x) { return (double)x.hi + (double)x.lo; }
__device__ __forceinline__ double to_double(double x) { return x; }
__device__ __forceinline__ float mag(dw x) { return fabsf(x.hi); }
__device__ __forceinline__ double mag(double x) { return fabs(x); }
__device__ __forceinline__ double to_double(float x) { return (double)x; }
__device__ __forceinline__ float mag(float x) { return fabsf(x); }
__device__ __forceinline__ dw dw_abs(dw x) { return x.hi < 0.0f ? -x : x; }
__device__ __forceinline__ dw dw_scale(dw x, float p2) { return dw{x.hi * p2, x.lo * p2}; }  // p2 = 2^k

// 1/sqrt(a) and 1/a of a double word a (a > 0 for the square root, a in the normal FP32 range):
// an FP32 seed r0 (2^-22 or better) and a Newton-Raphson step whose correction term
// e = 1 - a r0^2 (or 1 - a r0) is small, so it needs FP32 precision only and is evaluated with
// FMAs on the exact product r0^2.  That leaves 2^-46 for 1/x; 1/sqrt takes a second step in
// double words (the first leaves about 2^-44).
__device__ __forceinline__ dw dw_rsqrt(dw a) {
  const float r0 = rsqrtf(a.hi);
  const float p = __fmul_rn(r0, r0);
  const float pl = __fmaf_rn(r0, r0, -p);                 // r0^2 = p + pl exactly
  float e = __fmaf_rn(-a.hi, p, 1.0f);
  e = __fmaf_rn(-a.hi, pl, e);
  e = __fmaf_rn(-a.lo, p, e);
  const dw r1 = dw_fast_two_sum(r0, __fmul_rn(0.5f * r0, e));
  const dw e1 = dw_of(1.0f) - a * (r1 * r1);
  return r1 + dw_scale(r1 * dw_of(e1.hi), 0.5f);
}
__device__ __forceinline__ dw dw_rcp(dw a) {
  const float r0 = __frcp_rn(a.hi);
  float e = __fmaf_rn(-a.hi, r0, 1.0f);
  e = __fmaf_rn(-a.lo, r0, e);
  return dw_fast_two_sum(r0, __fmul_rn(r0, e));
}

// Householder reflector of house3 in double words.  (x, y, z) is first scaled by a power of two
// near 1 / max(|x|, |y|, |z|) so that no square under- or overflows FP32.
__device__ __forceinline__ void house3(dw x, dw y, dw z, dw& beta, dw& v1, dw& v2, dw& alpha) {
  const float amax = fmaxf(mag(x), fmaxf(mag(y), mag(z)));
  if ((mag(y) == 0.0f && mag(z) == 0.0f) || !(amax >= 1e-30f)) {   // nothing to annihilate
    beta = v1 = v2 = dw_of(0.0f);
    alpha = x;
    return;
  }
  // power-of-two scale from the exponent field (amax is a normal FP32 number here)
  const int ex = ((__float_as_int(amax) >> 23) & 0xff) - 127;
  const float f = __int_as_float((127 - ex) << 23), finv = __int_as_float((127 + ex) << 23);
  x = dw_scale(x, f);
  y = dw_scale(y, f);
  z = dw_scale(z, f);
  const dw n2 = x * x + (y * y + z * z);                 // in [1, 12)
  const dw rho = dw_rsqrt(n2);
  const dw mu = n2 * rho;
  const bool neg = x.hi < 0.0f;
  const dw v0 = neg ? x - mu : x + mu;
  const dw r = dw_rcp(v0);
  v1 = y * r;
  v2 = z * r;
  beta = dw_of(1.0f) + dw_abs(x) * rho;
  alpha = dw_scale(neg ? mu : -mu, finv);
}

// 3-vector (or 2-vector) Householder reflector P = I - beta v v^T, v = (1, v1, v2), with
// P (x, y, z)^T = (alpha, 0, 0)^T, alpha = -sign(x) ||(x, y, z)||.  With mu = ||(x, y, z)|| and
// v0 = x + sign(x) mu (no cancellation), v = (v0, y, z) / v0 and beta = 2 v0^2 / (v0^2 + y^2 + z^2)
// = 1 + |x| / mu, so one reciprocal square root and one reciprocal suffice.
__device__ __forceinline__ void house3(double x, double y, double z, double& beta, double& v1, double& v2,
                       double& alpha) {
  const double sigma = fma(z, z, y * y);
  if (sigma == 0.0) {
    beta = 0.0;
    v1 = v2 = 0.0;
    alpha = x;
    return;
  }
  const double n2 = fma(x, x, sigma);
  const double rho = rsqrt_nr(n2);
  const double mu = n2 * rho;
  const double s = (x < 0.0) ? -1.0 : 1.0;
  const double v0 = fma(s, mu, x);
  const double r = rcp_nr(v0);
  v1 = y * r;
  v2 = z * r;
  beta = fma(fabs(x), rho, 1.0);
  alpha = -s * mu;
}

struct Shared {
  double red[32];
  double scal[8];
  double shf[8];            // multi-bulge sweep: (sum, product) of each bulge's shift pair
  float hs[64];             // trailing block for the shifts (8 x 8, FP32)
  float hw[16];             // its eigenvalues (re 8 | im 8)
  int iscal[8];
  int sel_idx[kMaxKeep];
  int sel_part[kMaxKeep];   // 0 real, 1 real part of complex, 2 imaginary part of complex
  int job_q0[kMaxKeep];     // eigenvector jobs: selection entries [job_q0, job_q0 + job_len)
  int job_len[kMaxKeep];
  int out_pos[kMaxKeep];    // output position of each selection entry (ascending eigenvalues)
#ifdef BLM_EIG_TIMING
  long long msub[4];        // multi-bulge sweeps: window loads, chase, write-back, outside
  long long mphase[3];      // the chase's phases 0 (reflectors), 1 (rows), 2 (columns)
  long long msteps;         // the chase's time steps
#endif
};

// ---------------------------------------------------------------------------------------------
// Shifts of a multi-bulge sweep.  The 2 nb shifts are the eigenvalues of the trailing 2 nb x 2 nb
// block of the active window (the usual multishift choice), computed by one thread in FP32 with
// the plain Francis double-shift iteration: a shift only steers convergence, the sweep's
// accuracy does not depend on it.  They are paired from the bottom of the block upwards
// (complex conjugates together, real ones two by two) and each pair becomes one bulge's
// (sum, product).
// ---------------------------------------------------------------------------------------------
constexpr int kNbMax = 4;       // bulges chased together

__device__ __forceinline__ void house3f(float x, float y, float z, float& beta, float& v1, float& v2,
                        float& alpha) {
  const float sigma = fmaf(z, z, y * y);
  if (sigma == 0.0f) {
    beta = 0.0f;
    v1 = v2 = 0.0f;
    alpha = x;
    return;
  }
  // (the FP32 QR only locates eigenvalues, which FP64 inverse iteration recomputes: the
  // hardware reciprocal square root and approximate division, a few units in the last place,
  // keep this step's latency short)
  const float n2 = fmaf(x, x, sigma);
  const float rmu = rsqrtf(n2);
  const float mu = n2 * rmu;
  const float sg = x < 0.0f ? -1.0f : 1.0f;
  const float v0 = fmaf(sg, mu, x);
  const float rv0 = __fdividef(1.0f, v0);
  v1 = y * rv0;
  v2 = z * rv0;
  beta = fmaf(fabsf(x), rmu, 1.0f);
  alpha = -sg * mu;
}

__device__ __forceinline__ void house3(float x, float y, float z, float& beta, float& v1,
                                       float& v2, float& alpha) {
  house3f(x, y, z, beta, v1, v2, alpha);
}

// Eigenvalues of the n x n (n <= 8) Hessenberg matrix h (row-major, leading dimension 8), in
// place; false if the iteration does not converge.
__device__ bool small_eigs_f32(float* h, int n, float* wr, float* wi) {
  auto H = [&](int i, int j) -> float& { return h[i * 8 + j]; };
  int hi = n - 1, its = 0, total = 0;
  while (hi >= 0) {
    int l = hi;
    for (; l > 0; --l) {
      float s = fabsf(H(l - 1, l - 1)) + fabsf(H(l, l));
      if (s == 0.0f) s = 1.0f;
      if (fabsf(H(l, l - 1)) <= 1e-6f * s) break;   // shifts need no more
    }
    if (l == hi) {
      wr[hi] = H(hi, hi);
      wi[hi] = 0.0f;
      hi -= 1;
      its = 0;
      continue;
    }
    if (l == hi - 1) {
      const float a = H(hi - 1, hi - 1), b = H(hi - 1, hi), c = H(hi, hi - 1), d = H(hi, hi);
      const float p = 0.5f * (a - d), disc = p * p + b * c, mid = 0.5f * (a + d);
      if (disc >= 0.0f) {
        const float sq = sqrtf(disc);
        wr[hi - 1] = mid - sq;
        wr[hi] = mid + sq;
        wi[hi - 1] = wi[hi] = 0.0f;
      } else {
        const float sq = sqrtf(-disc);
        wr[hi - 1] = wr[hi] = mid;
        wi[hi - 1] = sq;
        wi[hi] = -sq;
      }
      hi -= 2;
      its = 0;
      continue;
    }
    if (++total > 30 * n) return false;
    ++its;
    float s, tt;
    if (its % 11 == 10) {
      const float e = fabsf(H(hi, hi - 1)) + fabsf(H(hi - 1, hi - 2));
      s = 1.5f * e;
      tt = e * e;
    } else {
      s = H(hi - 1, hi - 1) + H(hi, hi);
      tt = H(hi - 1, hi - 1) * H(hi, hi) - H(hi - 1, hi) * H(hi, hi - 1);
    }
    float x = H(l, l) * H(l, l) + H(l, l + 1) * H(l + 1, l) - s * H(l, l) + tt;
    float y = H(l + 1, l) * (H(l, l) + H(l + 1, l + 1) - s);
    float z = H(l + 1, l) * H(l + 2, l + 1);
    for (int k = l; k <= hi - 1; ++k) {
      const bool three = k <= hi - 2;
      if (k > l) {
        x = H(k, k - 1);
        y = H(k + 1, k - 1);
        z = three ? H(k + 2, k - 1) : 0.0f;
      }
      float beta, v1, v2, alpha;
      house3f(x, y, three ? z : 0.0f, beta, v1, v2, alpha);
      if (!three) v2 = 0.0f;
      if (beta == 0.0f) continue;
      if (k > l) {
        H(k, k - 1) = alpha;
        H(k + 1, k - 1) = 0.0f;
        if (three) H(k + 2, k - 1) = 0.0f;
      }
      for (int j = k; j <= hi; ++j) {
        const float p = H(k, j) + v1 * H(k + 1, j) + (three ? v2 * H(k + 2, j) : 0.0f);
        H(k, j) -= beta * p;
        H(k + 1, j) -= beta * v1 * p;
        if (three) H(k + 2, j) -= beta * v2 * p;
      }
      const int rmax = three ? min(k + 3, hi) : hi;
      for (int i = l; i <= rmax; ++i) {
        const float p = H(i, k) + v1 * H(i, k + 1) + (three ? v2 * H(i, k + 2) : 0.0f);
        H(i, k) -= beta * p;
        H(i, k + 1) -= beta * v1 * p;
        if (three) H(i, k + 2) -= beta * v2 * p;
      }
    }
  }
  return true;
}

// (sum, product) pairs for nb bulges from the n = 2 nb eigenvalues, bottom of the block first.
__device__ void pair_shifts(const float* wr, const float* wi, int n, int nb, double* shf) {
  int np = 0;
  bool have = false;
  double pend = 0.0;
  for (int i = n - 1; i >= 0 && np < nb;) {
    if (wi[i] != 0.0f && i > 0) {
      shf[2 * np] = 2.0 * (double)wr[i];
      shf[2 * np + 1] = (double)wr[i] * wr[i] + (double)wi[i] * wi[i];
      ++np;
      i -= 2;
    } else {
      if (have) {
        shf[2 * np] = pend + (double)wr[i];
        shf[2 * np + 1] = pend * (double)wr[i];
        ++np;
        have = false;
      } else {
        pend = wr[i];
        have = true;
      }
      i -= 1;
    }
  }
  for (int j = np; j < nb; ++j) {
    shf[2 * j] = np > 0 ? shf[0] : 0.0;
    shf[2 * j + 1] = np > 0 ? shf[1] : 0.0;
  }
}

// ---------------------------------------------------------------------------------------------
// Francis double-shift QR for all eigenvalues of the Hessenberg matrix G (dense, row-major
// m x m, global memory), FP64.  Only eigenvalues are wanted, so a sweep on the active window
// [l, hi] (l: last negligible subdiagonal) updates that window alone.
//
// A sweep's bulge is chased through square windows of at most kWin rows and columns held in
// shared memory.  Inside a window the first kChase threads run the steps: each computes the
// step's reflector from the bulge column itself (no broadcast), then applies it to the window's
// rows and columns, two barriers per step.  The parts of the same row and column operations
// that fall outside the window -- the window's rows right of it and its columns above it -- are
// applied after the window, from the stored reflectors, one thread per row or column with the
// three live entries in registers.  Every element receives the operations of the unwindowed
// sweep in the same order; the bulge column is set to (alpha, 0, 0) exactly.
// Returns false if the iteration budget (40 m sweeps) runs out.
// ---------------------------------------------------------------------------------------------
constexpr int kWin = 128;
constexpr int kWinLd = kWin + 1;
constexpr int kChase = 128;

__device__ __forceinline__ void chase_sync() {
  if (kChase == 32) {
    __syncwarp();
  } else {
    asm volatile("bar.sync 1, %0;" ::"n"(kChase) : "memory");
  }
}

// shared memory the QR needs: the window and the reflectors of one window (all bulges)
constexpr int kQrSmemDoubles = kWin * kWinLd + 4 * kWin * kNbMax;
static_assert(kChase == 32 * kNbMax, "one chase warp per bulge slot");
static_assert(kEigThreads == kNbMax * kWin, "one thread per (window row or column, bulge slot)");

// Arithmetic of the QR sweep: FP64, or double words (default; FP64 when it fails).
template <typename R>
struct QrArith;
template <>
struct QrArith<double> {
  static constexpr double kEps = 2.220446049250313e-16;   // deflation threshold (relative)
  __device__ static double of(double d) { return d; }
};
template <>
struct QrArith<float> {
  static constexpr double kEps = 3.0e-7;                  // about five FP32 units in the last place
  __device__ static float of(double d) { return (float)d; }
};
template <>
struct QrArith<dw> {
  static constexpr double kEps = 3.0e-14;                 // above the double-word rounding noise
  __device__ static dw of(double d) { return dw_of_double(d); }
};

// One QR sweep on the active window [l, hi] with nb (2..kNbMax) bulges chased together, their
// shift pairs in sh.shf.  Bulge j starts three steps after bulge j - 1 and, at time step tau,
// takes step k_j = l + tau - 3 j (active for l <= k_j <= hi - 1); bulges three rows apart touch
// disjoint rows in their row operations and disjoint columns in their column operations, so one
// time step applies all of them between barriers:
//   phase 0: warp j forms bulge j's reflector from its bulge column (or, at k_j = l, from the
//     shift polynomial's first column);
//   phase 1 (one thread per window column and bulge): the row operations;
//   phase 2 (one thread per window row and bulge): set the bulge column to (alpha, 0, 0) and
//     apply the column operations.  The one entry two bulges share -- row k_j + 3 of the
//     leading bulge's annihilated column, which the trailing bulge's column operation covers --
//     takes the leading bulge's alpha as the trailing operation's input and keeps the trailing
//     operation's result, as in the unpipelined order.
// Rows above and columns right of the window receive the same operations afterwards from the
// stored reflectors, all bulges of one time step on a sliding run of 3 kNbMax entries (their
// ranges are disjoint and adjacent), time steps in order.
// The w x w window at (a, a) of G into shared memory, four loads in flight per thread.
template <typename R>
__device__ __forceinline__ void load_window(const R* G, int m, int a, int w, R* win) {
  const int t = threadIdx.x, nt = blockDim.x, ww = w * w;
  for (int i0 = t; i0 < ww; i0 += 2 * nt) {
    R v[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int idx = i0 + u * nt;
      if (idx < ww) {
        const int r = idx / w, c = idx - r * w;
        v[u] = G[(int64_t)(a + r) * m + (a + c)];
      }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int idx = i0 + u * nt;
      if (idx < ww) {
        const int r = idx / w, c = idx - r * w;
        win[r * kWinLd + c] = v[u];
      }
    }
  }
}

template <typename R>
__device__ void multi_sweep(R* G, int m, int l, int hi, int nb, R* win, R* refl, Shared& sh) {
  using Q = QrArith<R>;
  const int t = threadIdx.x, nt = blockDim.x;
  const R zero = Q::of(0.0);
  auto g = [&](int i, int j) -> R& { return G[(int64_t)i * m + j]; };
  const int T = (hi - 1 - l) + 1 + 3 * (nb - 1);   // time steps of the sweep
  const int kSteps = kWin - 3 * kNbMax - 1;        // time steps per window
  for (int ts = 0; ts < T;) {
    const int te = min(ts + kSteps - 1, T - 1);
    const int a = max(l, l + ts - 3 * (nb - 1) - 1);   // window rows / columns a..b
    const int b = min(hi, l + te + 3);
    const int w = b - a + 1;
#ifdef BLM_EIG_TIMING
    long long tq = clock64();
#endif
    load_window(G, m, a, w, win);
    __syncthreads();
#ifdef BLM_EIG_TIMING
    if (t == 0) sh.msub[0] += clock64() - tq;
    tq = clock64();
#endif
    {
      auto W = [&](int i, int j) -> R& { return win[(i - a) * kWinLd + (j - a)]; };
      auto clampw = [&](int i) { return min(max(i, a), b); };
      // phases 1 and 2 run one thread per (column or row, slot): slot js = t / kWin of the
      // window's column or row a + (t mod kWin) (blockDim = kNbMax * kWin)
      const int js = t / kWin, tl = t - js * kWin;
      for (int tau = ts; tau <= te; ++tau) {
        R* rft = refl + (tau - ts) * kNbMax * 4;   // (beta, v1, v2, alpha) of each slot
#ifdef BLM_EIG_TIMING
        long long tp = clock64();
        if (t == 0) ++sh.msteps;
#endif
        if (t < kChase) {
          // phase 0: warp j forms slot j's reflector from its bulge column (or, at k = l, from
          // the shift polynomial's first column)
          const int j = t >> 5;
          const int k = l + tau - 3 * j;
          R be = zero, w1 = zero, w2 = zero, al = zero;
          if (j < nb && k >= l && k <= hi - 1) {
            const bool three = k <= hi - 2;
            R x, y, z;
            if (k == l) {
              const R s = Q::of(sh.shf[2 * j]), tt = Q::of(sh.shf[2 * j + 1]);
              const R h00 = W(l, l), h10 = W(l + 1, l), h01 = W(l, l + 1);
              const R h11 = W(l + 1, l + 1), h21 = W(l + 2, l + 1);
              x = h00 * h00 + h01 * h10 - s * h00 + tt;
              y = h10 * (h00 + h11 - s);
              z = h10 * h21;
            } else {
              x = W(k, k - 1);
              y = W(k + 1, k - 1);
              z = three ? W(k + 2, k - 1) : zero;
            }
            house3(x, y, three ? z : zero, be, w1, w2, al);
            if (!three) w2 = zero;
          }
          if ((t & 31) == 0) {
            rft[4 * j] = be;
            rft[4 * j + 1] = w1;
            rft[4 * j + 2] = w2;
            rft[4 * j + 3] = al;
          }
        }
        __syncthreads();
#ifdef BLM_EIG_TIMING
        if (t == 0) sh.mphase[0] += clock64() - tp;
        tp = clock64();
#endif
        const int k = l + tau - 3 * js;
        const R be = rft[4 * js], v1 = rft[4 * js + 1], v2 = rft[4 * js + 2], al = rft[4 * js + 3];
        const bool act = js < nb && k >= l && k <= hi - 1 && mag(be) != 0;
        const R bv1 = be * v1, bv2 = be * v2;
        const bool three = k <= hi - 2;
        // phase 1: row operations of slot js on column c (the slots' rows are disjoint)
        {
          const int c = a + tl;
          if (act && c <= b && c >= k) {
            const R r0 = W(k, c), r1 = W(k + 1, c), r2 = three ? W(k + 2, c) : zero;
            const R p = r0 + (v1 * r1 + v2 * r2);
            W(k, c) = r0 - be * p;
            W(k + 1, c) = r1 - bv1 * p;
            if (three) W(k + 2, c) = r2 - bv2 * p;
          }
        }
        __syncthreads();
#ifdef BLM_EIG_TIMING
        if (t == 0) sh.mphase[1] += clock64() - tp;
        tp = clock64();
#endif
        // phase 2: slot js's bulge column and column operations on row r.  Column k + 2 is the
        // leading slot's (js - 1) annihilated bulge column: on its row k + 3 that slot's alpha
        // enters this operation, and this slot's result is what the entry keeps (the leading
        // slot leaves its alpha unwritten there).
        {
          const int r = a + tl;
          if (act && r <= b) {
            const int kt = k - 3;   // the trailing slot (js + 1)
            bool trail = false;
            if (js + 1 < nb && kt >= l) {
              const R bt = rft[4 * (js + 1)];
              trail = mag(bt) != 0 && kt <= hi - 2;
            }
            if (k > l && r >= k && r <= k + (three ? 2 : 1) && !(r == k && trail))
              W(r, k - 1) = (r == k) ? al : zero;
            const int rmax = three ? min(k + 3, hi) : hi;
            if (r <= rmax) {
              const R c0 = W(r, k), c1 = W(r, k + 1);
              R c2 = three ? W(r, k + 2) : zero;
              if (js > 0 && three && r == k + 3) {
                const int kl = k + 3;   // the leading slot's step
                const R bl = rft[4 * (js - 1)];
                if (kl <= hi - 1 && mag(bl) != 0) c2 = rft[4 * (js - 1) + 3];
              }
              const R p = c0 + (v1 * c1 + v2 * c2);
              W(r, k) = c0 - be * p;
              W(r, k + 1) = c1 - bv1 * p;
              if (three) W(r, k + 2) = c2 - bv2 * p;
            }
          }
        }
        __syncthreads();
#ifdef BLM_EIG_TIMING
        if (t == 0) sh.mphase[2] += clock64() - tp;
#endif
      }
    }
    __syncthreads();
#ifdef BLM_EIG_TIMING
    if (t == 0) sh.msub[1] += clock64() - tq;
    tq = clock64();
#endif
    for (int idx = t; idx < w * w; idx += nt) {
      const int r = idx / w, c = idx - r * w;
      g(a + r, a + c) = win[r * kWinLd + c];
    }
#ifdef BLM_EIG_TIMING
    __syncthreads();
    if (t == 0) sh.msub[2] += clock64() - tq;
    tq = clock64();
#endif
    // rows l..a-1 (column operations, walking right) and columns b+1..hi (row operations,
    // walking down); entry i of the run is position p0 + i, bulge j on entries 9-3j..11-3j
    const int nfa = a - l, nfb = hi - b;
    for (int u = t; u < nfa + nfb; u += nt) {
      const bool row_walk = u < nfa;
      const int64_t base = row_walk ? (int64_t)(l + u) * m : (int64_t)(b + 1 + u - nfa);
      const int64_t step = row_walk ? 1 : m;
      auto ld = [&](int e) { return (e >= a && e <= b) ? G[base + (int64_t)e * step] : zero; };
      auto st = [&](int e, const R& v) {
        if (e >= a && e <= b) G[base + (int64_t)e * step] = v;
      };
      int p0 = l + ts - 3 * (kNbMax - 1);
      R e[3 * kNbMax], q[4];
#pragma unroll
      for (int i = 0; i < 3 * kNbMax; ++i) e[i] = ld(p0 + i);
#pragma unroll
      for (int i = 0; i < 4; ++i) q[i] = ld(p0 + 3 * kNbMax + i);
      for (int tau = ts; tau <= te; ++tau) {
        const R* rf = refl + (tau - ts) * kNbMax * 4;
#pragma unroll
        for (int j = 0; j < kNbMax; ++j) {
          // inactive slots carry beta = 0 and leave their entries unchanged exactly
          const R beta = rf[4 * j], w1 = rf[4 * j + 1], w2 = rf[4 * j + 2];
          R& x0 = e[3 * (kNbMax - 1 - j)];
          R& x1 = e[3 * (kNbMax - 1 - j) + 1];
          R& x2 = e[3 * (kNbMax - 1 - j) + 2];
          const R p = x0 + (w1 * x1 + w2 * x2);
          x0 = x0 - beta * p;
          x1 = x1 - (beta * w1) * p;
          x2 = x2 - (beta * w2) * p;
        }
        st(p0, e[0]);
#pragma unroll
        for (int i = 0; i < 3 * kNbMax - 1; ++i) e[i] = e[i + 1];
        e[3 * kNbMax - 1] = q[0];
        q[0] = q[1];
        q[1] = q[2];
        q[2] = q[3];
        q[3] = ld(p0 + 3 * kNbMax + 4);
        ++p0;
      }
#pragma unroll
      for (int i = 0; i < 3 * kNbMax; ++i) st(p0 + i, e[i]);
    }
    __syncthreads();
#ifdef BLM_EIG_TIMING
    if (t == 0) sh.msub[3] += clock64() - tq;
#endif
    ts = te + 1;
  }
}

template <typename R>
__device__ bool hqr_windowed(R* G, int m, double* wr, double* wi, double anorm, double* dsm,
                             Shared& sh) {
  using Q = QrArith<R>;
  const int t = threadIdx.x, nt = blockDim.x;
  const double eps = Q::kEps;
  R* win = reinterpret_cast<R*>(dsm);
  R* refl = win + kWin * kWinLd;
  const R zero = Q::of(0.0);
  int hi = m - 1;
  int its = 0, total = 0;
  const int limit = 40 * m + 100;
  auto g = [&](int i, int j) -> R& { return G[(int64_t)i * m + j]; };
#ifdef BLM_EIG_TIMING
  long long qt[4] = {0, 0, 0, 0}, qc = 0, nsweep = 0, nstep = 0, nmulti = 0, nsfail = 0;
  if (t == 0) {
    sh.msub[0] = sh.msub[1] = sh.msub[2] = sh.msub[3] = 0;
    sh.mphase[0] = sh.mphase[1] = sh.mphase[2] = sh.msteps = 0;
  }
#define QR_T0() (qc = clock64())
#define QR_T(i) (qt[i] += clock64() - qc, qc = clock64())
#else
#define QR_T0() ((void)0)
#define QR_T(i) ((void)0)
#endif
  while (hi >= 0) {
    QR_T0();
    // --- deflation: the largest i in [1, hi] whose subdiagonal entry is negligible ---
    if (t == 0) sh.iscal[0] = 0;
    __syncthreads();
    for (int i = hi - t; i >= 1; i -= nt) {
      double s = (double)mag(g(i - 1, i - 1)) + (double)mag(g(i, i));
      if (s == 0.0) s = anorm;
      if ((double)mag(g(i, i - 1)) <= eps * s) {
        atomicMax(&sh.iscal[0], i);
        break;
      }
    }
    __syncthreads();
    const int l = sh.iscal[0];
    if (l == hi || l == hi - 1) {
      if (t == 0) {
        if (l > 0) g(l, l - 1) = zero;
        if (l == hi) {
          wr[hi] = to_double(g(hi, hi));
          wi[hi] = 0.0;
        } else {
          const double a = to_double(g(hi - 1, hi - 1)), b = to_double(g(hi - 1, hi));
          const double c = to_double(g(hi, hi - 1)), d = to_double(g(hi, hi));
          const double p = 0.5 * (a - d);
          const double disc = p * p + b * c;
          const double mid = 0.5 * (a + d);
          if (disc >= 0.0) {
            const double s = sqrt(disc);
            const double l1 = mid + (mid >= 0.0 ? s : -s);
            double l2 = mid - (mid >= 0.0 ? s : -s);
            const double det = a * d - b * c;
            if (l1 != 0.0) l2 = det / l1;
            wr[hi - 1] = fmin(l1, l2);
            wr[hi] = fmax(l1, l2);
            wi[hi - 1] = wi[hi] = 0.0;
          } else {
            const double s = sqrt(-disc);
            wr[hi - 1] = wr[hi] = mid;
            wi[hi - 1] = s;
            wi[hi] = -s;
          }
        }
      }
      hi -= (l == hi) ? 1 : 2;
      its = 0;
      __syncthreads();
      continue;
    }
    if (total >= limit) return false;
    ++its;
    ++total;
#ifdef BLM_EIG_TIMING
    ++nsweep;
    nstep += hi - l;
#endif
    const int nact = hi - l + 1;
    const int nb = (its % 11 == 10) ? 1 : (nact >= 40 ? kNbMax : (nact >= 20 ? 2 : 1));
#ifdef BLM_EIG_TIMING
    nstep += (long long)(nb - 1) * (hi - l);   // bulge steps
#endif
    if (nb > 1) {
      // --- multi-bulge sweep: shifts from the trailing 2 nb x 2 nb block (thread 0) ---
      if (t == 0) {
        if (l > 0) g(l, l - 1) = zero;
        const int n = 2 * nb, o = hi - n + 1;
        for (int i = 0; i < n; ++i)
          for (int j = 0; j < n; ++j)
            sh.hs[i * 8 + j] = (j >= i - 1) ? (float)to_double(g(o + i, o + j)) : 0.0f;
#ifdef BLM_EIG_TIMING
        ++nmulti;
#endif
        if (small_eigs_f32(sh.hs, n, sh.hw, sh.hw + 8)) {
          pair_shifts(sh.hw, sh.hw + 8, n, nb, sh.shf);
          // the leading bulge takes the Francis shifts of the trailing 2 x 2 in full precision
          sh.shf[0] = to_double(g(hi - 1, hi - 1) + g(hi, hi));
          sh.shf[1] = to_double(g(hi - 1, hi - 1) * g(hi, hi) - g(hi - 1, hi) * g(hi, hi - 1));
        } else {
#ifdef BLM_EIG_TIMING
          ++nsfail;
#endif
          // the trailing 2 x 2 diagonal blocks' eigenvalues
          for (int j = 0; j < nb; ++j) {
            const int i0 = hi - 2 * j - 1;
            sh.shf[2 * j] = to_double(g(i0, i0) + g(i0 + 1, i0 + 1));
            sh.shf[2 * j + 1] = to_double(g(i0, i0) * g(i0 + 1, i0 + 1) - g(i0, i0 + 1) * g(i0 + 1, i0));
          }
        }
      }
      __syncthreads();
      QR_T(0);
      multi_sweep<R>(G, m, l, hi, nb, win, refl, sh);
      QR_T(2);
      continue;
    }
    // --- shifts and the first column of the double-shift polynomial (thread 0) ---
    if (t == 0) {
      if (l > 0) g(l, l - 1) = zero;
      R s, tt;
      if (its % 11 == 10) {
        const R e = Q::of((double)mag(g(hi, hi - 1)) + (double)mag(g(hi - 1, hi - 2)));
        s = Q::of(1.5) * e;
        tt = e * e;
      } else {
        s = g(hi - 1, hi - 1) + g(hi, hi);
        tt = g(hi - 1, hi - 1) * g(hi, hi) - g(hi - 1, hi) * g(hi, hi - 1);
      }
      const R h00 = g(l, l), h10 = g(l + 1, l), h01 = g(l, l + 1);
      const R h11 = g(l + 1, l + 1), h21 = g(l + 2, l + 1);
      const R x0 = h00 * h00 + h01 * h10 - s * h00 + tt;
      const R y0 = h10 * (h00 + h11 - s);
      const R z0 = h10 * h21;
      sh.scal[0] = to_double(x0);
      sh.scal[1] = to_double(y0);
      sh.scal[2] = to_double(z0);
    }
    __syncthreads();
    QR_T(0);
    // --- the sweep, window by window ---
    for (int ks = l; ks <= hi - 1;) {
      const int ke = min(ks + kWin - 5, hi - 1);   // steps ks..ke in this window
      const int a = (ks > l) ? ks - 1 : l;         // window rows/columns a..b
      const int b = min(ke + 3, hi);
      const int w = b - a + 1;
      load_window(G, m, a, w, win);
      __syncthreads();
      QR_T(1);
      if (t < kChase) {
        auto W = [&](int i, int j) -> R& { return win[(i - a) * kWinLd + (j - a)]; };
        for (int k = ks; k <= ke; ++k) {
          const bool three = (k <= hi - 2);
          R x, y, z;
          if (k == l) {
            x = Q::of(sh.scal[0]);
            y = Q::of(sh.scal[1]);
            z = Q::of(sh.scal[2]);
          } else {
            x = W(k, k - 1);
            y = W(k + 1, k - 1);
            z = three ? W(k + 2, k - 1) : zero;
          }
          R beta, v1, v2, alpha;
          house3(x, y, three ? z : zero, beta, v1, v2, alpha);
          if (!three) v2 = zero;
          const R bv1 = beta * v1, bv2 = beta * v2;
          const bool act = mag(beta) != 0;
          if (t == 0) {
            refl[3 * (k - ks)] = beta;
            refl[3 * (k - ks) + 1] = v1;
            refl[3 * (k - ks) + 2] = v2;
          }
          if (act) {
            // rows k..k+2, columns k..b (the bulge column k-1 is set below)
            for (int j = k + t; j <= b; j += kChase) {
              R& r0 = W(k, j);
              R& r1 = W(k + 1, j);
              if (three) {
                R& r2 = W(k + 2, j);
                const R p = r0 + (v1 * r1 + v2 * r2);
                r0 = r0 - beta * p;
                r1 = r1 - bv1 * p;
                r2 = r2 - bv2 * p;
              } else {
                const R p = r0 + v1 * r1;
                r0 = r0 - beta * p;
                r1 = r1 - bv1 * p;
              }
            }
          }
          chase_sync();   // every thread has read the bulge column and finished its rows
          if (act) {
            if (t == 0 && k > l) {
              W(k, k - 1) = alpha;
              W(k + 1, k - 1) = zero;
              if (three) W(k + 2, k - 1) = zero;
            }
            // columns k..k+2, rows a..min(k+3, hi)
            const int rmax = three ? min(k + 3, hi) : hi;
            for (int i = a + t; i <= rmax; i += kChase) {
              R& c0 = W(i, k);
              R& c1 = W(i, k + 1);
              if (three) {
                R& c2 = W(i, k + 2);
                const R p = c0 + (v1 * c1 + v2 * c2);
                c0 = c0 - beta * p;
                c1 = c1 - bv1 * p;
                c2 = c2 - bv2 * p;
              } else {
                const R p = c0 + v1 * c1;
                c0 = c0 - beta * p;
                c1 = c1 - bv1 * p;
              }
            }
          }
          chase_sync();
        }
      }
      __syncthreads();
      QR_T(2);
      for (int idx = t; idx < w * w; idx += nt) {
        const int r = idx / w, c = idx - r * w;
        g(a + r, a + c) = win[r * kWinLd + c];
      }
      // operations outside the window: columns ks..ke+2 of rows l..a-1 (column operations) and
      // rows ks..ke+2 of columns b+1..hi (row operations)
      const int nfa = a - l, nfb = hi - b;
      for (int u = t; u < nfa + nfb; u += nt) {
        // a row above the window walks right along its columns; a column right of the window
        // walks down its rows: element e of the walk is G[base + e * step]
        const bool row_walk = u < nfa;
        const int64_t base = row_walk ? (int64_t)(l + u) * m : (int64_t)(b + 1 + u - nfa);
        const int64_t step = row_walk ? 1 : m;
        // e0..e2: positions k..k+2; q0..q3: positions k+3..k+6 loaded ahead (L2 latency)
        auto ld = [&](int e) { return (e <= hi) ? G[base + (int64_t)e * step] : zero; };
        R e0 = ld(ks), e1 = ld(ks + 1), e2 = ld(ks + 2);
        R q0 = ld(ks + 3), q1 = ld(ks + 4), q2 = ld(ks + 5), q3 = ld(ks + 6);
        for (int k = ks; k <= ke; ++k) {
          const R beta = refl[3 * (k - ks)];
          if (mag(beta) != 0) {
            const R v1 = refl[3 * (k - ks) + 1], v2 = refl[3 * (k - ks) + 2];
            const R p = e0 + (v1 * e1 + v2 * e2);   // v2 = 0 on the last (two-row) step
            e0 = e0 - beta * p;
            e1 = e1 - (beta * v1) * p;
            e2 = e2 - (beta * v2) * p;
          }
          G[base + (int64_t)k * step] = e0;
          e0 = e1;
          e1 = e2;
          e2 = q0;
          q0 = q1;
          q1 = q2;
          q2 = q3;
          q3 = ld(k + 7);
        }
        if (ke + 1 <= hi) G[base + (int64_t)(ke + 1) * step] = e0;
        if (ke + 2 <= hi) G[base + (int64_t)(ke + 2) * step] = e1;
      }
      __syncthreads();
      QR_T(3);
      ks = ke + 1;
    }
  }
#ifdef BLM_EIG_TIMING
  if (t == 0 && blockIdx.x == 0)
    printf("qr m=%d sweeps %lld (multi-bulge %lld, shift failures %lld) steps %lld: deflate+shift %lld "
           "window-load %lld chase %lld far %lld cycles\n",
           m, nsweep, nmulti, nsfail, nstep, qt[0], qt[1], qt[2], qt[3]);
  if (t == 0)
    printf("qr m=%d multi-bulge sweeps: window loads %lld chase %lld write-back %lld outside %lld cycles; "
           "%lld time steps: reflectors %lld rows %lld columns %lld cycles\n",
           m, sh.msub[0], sh.msub[1], sh.msub[2], sh.msub[3], sh.msteps, sh.mphase[0], sh.mphase[1],
           sh.mphase[2]);
#endif
#undef QR_T0
#undef QR_T
  return true;
}

// ---------------------------------------------------------------------------------------------
// Per-warp inverse iteration on the FP64 Hessenberg matrix Hh (no CTA barriers): one warp
// factors (Hh - sigma I) = P L U with the one-row pivoting a Hessenberg matrix needs and solves
// with the factors.  Rows being eliminated live in shared memory (cur, nxt); U is stored packed
// (row k holds columns k..m-1).  CX selects complex arithmetic (complex shift) at compile time.
// ---------------------------------------------------------------------------------------------
constexpr int kVecWarps = 16;                          // warps of a CTA running inverse iteration
constexpr int kVecSlots = 32;                          // factor slots of a problem (its team's warps)
constexpr int kEigSmemDoubles = 200 * 1024 / 8;        // dynamic shared memory of the solver
static_assert(kQrSmemDoubles <= kEigSmemDoubles, "QR window exceeds the solver's shared memory");

// Workspace of dense_geig for dimension m: L, A, Hh (m^2 each), W (2 m^2), 6 vectors of m;
// then the per-warp factors and pivots and the kMaxKeep Hessenberg-basis eigenvectors.
__host__ __device__ constexpr int64_t eig_base_doubles(int64_t m) { return 5 * m * m + 6 * m; }
constexpr int kMaxTeam = 8;                             // CTAs per problem at most
// the end of the eigenvector section
__host__ __device__ constexpr int64_t eig_rank_offset(int64_t m) {
  return eig_base_doubles(m) + kVecSlots * m * (m + 1) + kVecSlots * 3 * m + kMaxKeep * 2 * m;
}
__host__ __device__ constexpr int64_t eig_total_doubles(int64_t m) {
  return eig_rank_offset(m) + 64;
}

__device__ __forceinline__ int64_t urow(int k, int m) {
  return (int64_t)k * m - ((int64_t)k * (k - 1)) / 2;
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// (Hh - sigma I) = P L U by one warp, Hessenberg pivoting; U packed by rows into U.
template <bool CX>
__device__ void warp_hess_lu(const double* Hh, int m, double s_re, double s_im, double pert,
                             double* cur, double* nxt, double* U, double* pl, int* ps) {
  const int lane = threadIdx.x & 31;
  const int64_t half = (int64_t)m * (m + 1) / 2;
  for (int j = lane; j < m; j += 32) {
    cur[j] = Hh[j] - (j == 0 ? s_re : 0.0);
    if (CX) cur[m + j] = (j == 0) ? -s_im : 0.0;
  }
  __syncwarp();
  for (int k = 0; k < m - 1; ++k) {
    const double* hrow = Hh + (int64_t)(k + 1) * m;
    for (int j = k + lane; j < m; j += 32) {
      nxt[j] = hrow[j] - (j == k + 1 ? s_re : 0.0);
      if (CX) nxt[m + j] = (j == k + 1) ? -s_im : 0.0;
    }
    __syncwarp();
    cplx a = cmk(cur[k], CX ? cur[m + k] : 0.0), b = cmk(nxt[k], CX ? nxt[m + k] : 0.0);
    const int sw = cabs2(b) > cabs2(a) ? 1 : 0;
    if (sw) {
      const cplx tmp = a;
      a = b;
      b = tmp;
    }
    if (cabs2(a) == 0.0) a = cmk(pert, 0.0);
    const cplx lm = CX ? cdiv(b, a) : cmk(b.re * rcp_nr(a.re), 0.0);
    __syncwarp();   // every lane has read row k before it is overwritten
    double* urk = U + urow(k, m) - k;
    for (int j = k + lane; j < m; j += 32) {
      const double cr = cur[j], nr = nxt[j];
      const double ci = CX ? cur[m + j] : 0.0, ni = CX ? nxt[m + j] : 0.0;
      const double tr = sw ? nr : cr, ti = sw ? ni : ci;
      const double br = sw ? cr : nr, bi = sw ? ci : ni;
      urk[j] = tr;
      if (CX) urk[half + j] = ti;
      cur[j] = br - (lm.re * tr - lm.im * ti);
      if (CX) cur[m + j] = bi - (lm.re * ti + lm.im * tr);
    }
    if (lane == 0) {
      pl[k] = lm.re;
      pl[m + k] = lm.im;
      ps[k] = sw;
    }
    __syncwarp();
  }
  if (lane == 0) {
    U[urow(m - 1, m)] = cur[m - 1];
    if (CX) U[half + urow(m - 1, m)] = cur[2 * m - 1];
  }
  __syncwarp();
}

// One solve with the factors of warp_hess_lu, in place (y: re [0, m), im [m, 2m) when CX),
// then scaling to max-abs 1.
template <bool CX>
__device__ void warp_hess_solve(int m, double pert, const double* U, const double* pl,
                                const int* ps, double* y) {
  const int lane = threadIdx.x & 31;
  const int64_t half = (int64_t)m * (m + 1) / 2;
  if (lane == 0) {
    for (int k = 0; k < m - 1; ++k) {
      cplx a = cmk(y[k], CX ? y[m + k] : 0.0), b = cmk(y[k + 1], CX ? y[m + k + 1] : 0.0);
      if (ps[k]) {
        const cplx tmp = a;
        a = b;
        b = tmp;
      }
      b = b - cmk(pl[k], CX ? pl[m + k] : 0.0) * a;
      y[k] = a.re;
      y[k + 1] = b.re;
      if (CX) {
        y[m + k] = a.im;
        y[m + k + 1] = b.im;
      }
    }
  }
  __syncwarp();
  for (int k = m - 1; k >= 0; --k) {
    const double* urk = U + urow(k, m) - k;
    double sr = 0.0, si = 0.0;
    for (int j = k + 1 + lane; j < m; j += 32) {
      const double ur = urk[j], xr = y[j];
      if (CX) {
        const double ui = urk[half + j], xi = y[m + j];
        sr += ur * xr - ui * xi;
        si += ur * xi + ui * xr;
      } else {
        sr = fma(ur, xr, sr);
      }
    }
    sr = warp_sum(sr);
    if (CX) si = warp_sum(si);
    if (lane == 0) {
      cplx d = cmk(urk[k], CX ? urk[half + k] : 0.0);
      if (cabs2(d) == 0.0) d = cmk(pert, 0.0);
      const cplx num = cmk(y[k] - sr, CX ? y[m + k] - si : 0.0);
      const cplx x = CX ? cdiv(num, d) : cmk(num.re * rcp_nr(d.re), 0.0);
      y[k] = x.re;
      if (CX) y[m + k] = x.im;
    }
    __syncwarp();
  }
  double mx = 0.0;
  for (int i = lane; i < m; i += 32) mx = fmax(mx, fabs(y[i]) + (CX ? fabs(y[m + i]) : 0.0));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const double inv = mx > 0.0 ? 1.0 / mx : 1.0;
  for (int i = lane; i < m; i += 32) {
    y[i] *= inv;
    if (CX) y[m + i] *= inv;
  }
  __syncwarp();
}

__device__ double warp_dot(const double* a, const double* b, int m) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int i = lane; i < m; i += 32) s = fma(a[i], b[i], s);
  return warp_sum(s);
}

// Per-warp v <- D L^-T Q v for a real vector v (in shared memory).  Rt holds the Householder
// vectors of the Hessenberg reduction as rows (Rt[k][i] = A[i][k], i >= k + 2).
__device__ void warp_back_transform(const double* Rt, const double* hbeta, const double* L,
                                    const double* dsc, int m, double* v) {
  const int lane = threadIdx.x & 31;
  for (int k = m - 3; k >= 0; --k) {
    const double beta = hbeta[k];
    if (beta == 0.0) continue;
    const double* u = Rt + (int64_t)k * m;
    double part = 0.0;
    for (int i = k + 1 + lane; i < m; i += 32) part = fma(i == k + 1 ? 1.0 : u[i], v[i], part);
    const double dot = beta * warp_sum(part);
    __syncwarp();
    for (int i = k + 1 + lane; i < m; i += 32) v[i] -= dot * (i == k + 1 ? 1.0 : u[i]);
    __syncwarp();
  }
  for (int i = m - 1; i >= 0; --i) {
    const double* li = L + (int64_t)i * m;
    const double zi = v[i] / li[i];
    __syncwarp();
    if (lane == 0) v[i] = zi;
    for (int j = lane; j < i; j += 32) v[j] -= li[j] * zi;
    __syncwarp();
  }
  for (int i = lane; i < m; i += 32) v[i] *= dsc[i];
  __syncwarp();
}


// Phase timing of dense_geig (debug builds with -DBLM_EIG_TIMING): clock64 marks printed by
// thread 0 of the first problem of a launch.
#ifdef BLM_EIG_TIMING
#define EIG_MARK(i)                                  \
  do {                                               \
    if (threadIdx.x == 0) tmark[i] = clock64();      \
  } while (0)
#else
#define EIG_MARK(i) \
  do {              \
  } while (0)
#endif

// Row kernels of the dense reductions, lanes over columns.  Small matrices (the Davidson
// projection, m <= 64) go one row per warp; larger ones four rows per warp (below).
// a[j] -= s * x[j], j = j0 + lane, j0 + lane + 32, ... < j1
__device__ __forceinline__ void row_axpy(double* __restrict__ a, const double* __restrict__ x,
                                         double s, int j0, int j1, int lane) {
#pragma unroll 4
  for (int j = j0 + lane; j < j1; j += 32) a[j] -= s * x[j];
}
// sum over j of a[j] * x[j] (this lane's part)
__device__ __forceinline__ double row_dot(const double* __restrict__ a, const double* __restrict__ x,
                                          int j0, int j1, int lane) {
  double s0 = 0.0, s1 = 0.0;
  int j = j0 + lane;
  for (; j + 32 < j1; j += 64) {
    s0 = fma(a[j], x[j], s0);
    s1 = fma(a[j + 32], x[j + 32], s1);
  }
  if (j < j1) s0 = fma(a[j], x[j], s0);
  return s0 + s1;
}
constexpr int kRows4Min = 64;   // matrices larger than this use the four-row kernels

// Four-row kernels.
// Four rows i_r = i0 + r * stride (those below iend) of a row-major matrix with leading
// dimension ld, by one warp: a_i[j] -= s_r * x[j] for j in [j0, j1_r).  The matrices live in
// global memory (L2), so each 128-column chunk's loads of all four rows are issued before any
// store: sixteen loads in flight per lane instead of the four of a single row.
__device__ __forceinline__ void rows4_axpy(double* a, int64_t ld, int i0, int stride, int iend,
                                           const double* s, const int* j1, const double* x,
                                           int j0, int lane) {
  int jmax = j0;
#pragma unroll
  for (int r = 0; r < 4; ++r)
    if (i0 + r * stride < iend) jmax = max(jmax, j1[r]);
  for (int jc = j0 + lane; jc < jmax; jc += 128) {
    double v[4][4], xv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) xv[q] = (jc + 32 * q < jmax) ? x[jc + 32 * q] : 0.0;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = i0 + r * stride, j = jc + 32 * q;
        v[r][q] = (i < iend && j < j1[r]) ? a[(int64_t)i * ld + j] : 0.0;
      }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = i0 + r * stride, j = jc + 32 * q;
        if (i < iend && j < j1[r]) a[(int64_t)i * ld + j] = v[r][q] - s[r] * xv[q];
      }
  }
}

// The same four rows: z_r = a_i . x over [j0, j1), then a_i[j] -= beta z_r x[j].
__device__ __forceinline__ void rows4_dot_axpy(double* a, int64_t ld, int i0, int stride, int iend,
                                               const double* x, double beta, int j0, int j1,
                                               int lane) {
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int jc = j0 + lane; jc < j1; jc += 128) {
    double xv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) xv[q] = (jc + 32 * q < j1) ? x[jc + 32 * q] : 0.0;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = i0 + r * stride, j = jc + 32 * q;
        const double v = (i < iend && j < j1) ? a[(int64_t)i * ld + j] : 0.0;
        acc[r] = fma(v, xv[q], acc[r]);
      }
  }
  double sc[4];
  int j1r[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    for (int o = 16; o > 0; o >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
    sc[r] = beta * acc[r];
    j1r[r] = j1;
  }
  rows4_axpy(a, ld, i0, stride, iend, sc, j1r, x, j0, lane);
}


// ---------------------------------------------------------------------------------------------
// Teams: one problem solved by T CTAs of a cooperative launch (all resident), which meet at a
// bounded barrier on a per-problem control block in global memory (zeroed before the launch).
// A wait that runs out marks the block, and every rank then gives up at its next barrier.
// ---------------------------------------------------------------------------------------------
constexpr uint32_t kTeamSpinLimit = 1u << 26;
struct TeamCtl {
  unsigned int count, gen;  // barrier arrivals, generation
  int err;                  // a barrier gave up
  int flag;                 // a rank's early status (ST_*), read after a barrier
  int qr_ok;                // rank 0's QR: 1 located in FP32, 2 in double words or FP64, 0 failed
  int vec_fail;             // an eigenvector that is no eigenvector (double-word location)
  unsigned long long anorm_bits;   // max |Hessenberg entry| as the bits of a non-negative double
  double sel_err[kMaxKeep]; // FP32 location: |FP64 quotient - FP32 value| per kept entry
  double sel_qim[kMaxKeep]; // and the FP64 quotient's imaginary part (complex entries)
};
struct Team {
  int r, T;
  TeamCtl* ctl;
};

__device__ bool team_sync(const Team& tm, TeamCtl* c, int* ok_smem) {
  __syncthreads();
  if (tm.T == 1) return true;
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = &c->gen;
    const unsigned int g = *vgen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(&c->count, 1u) == (unsigned int)tm.T - 1) {
      atomicExch(&c->count, 0u);
      __threadfence();
      atomicAdd(&c->gen, 1u);
    } else {
      uint32_t i = 0;
      while (*vgen == g) {
        if (++i > kTeamSpinLimit || *(volatile int*)&c->err) {
          ok = 0;
          atomicExch(&c->err, 1);
          break;
        }
        __nanosleep(32);
      }
    }
    if (*(volatile int*)&c->err) ok = 0;
    __threadfence();
    *ok_smem = ok;
  }
  __syncthreads();
  return *ok_smem != 0;
}

// Column pieces of 32: piece p belongs to rank p mod T.  The first piece of rank R that holds a
// column >= j0.
__device__ __forceinline__ int first_piece(int j0, int R, int T) {
  const int p = j0 >> 5;
  return p + ((R - p) % T + T) % T;
}
// a[j] -= s * x[j] for this rank's columns j in [j0, j1)
__device__ __forceinline__ void row_axpy_own(double* __restrict__ a, const double* __restrict__ x,
                                             double s, int j0, int j1, int lane, int R, int T) {
  for (int p = first_piece(j0, R, T); 32 * p < j1; p += T) {
    const int j = 32 * p + lane;
    if (j >= j0 && j < j1) a[j] -= s * x[j];
  }
}
// rows4_axpy over this rank's column pieces (four pieces per pass; T = 1: 128 contiguous columns)
__device__ __forceinline__ void rows4_axpy_own(double* a, int64_t ld, int i0, int stride, int iend,
                                               const double* s, const int* j1, const double* x,
                                               int j0, int lane, int R, int T) {
  int jmax = j0;
#pragma unroll
  for (int r = 0; r < 4; ++r)
    if (i0 + r * stride < iend) jmax = max(jmax, j1[r]);
  for (int p = first_piece(j0, R, T); 32 * p < jmax; p += 4 * T) {
    double v[4][4], xv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = 32 * (p + q * T) + lane;
      xv[q] = (j >= j0 && j < jmax) ? x[j] : 0.0;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = i0 + r * stride, j = 32 * (p + q * T) + lane;
        v[r][q] = (i < iend && j >= j0 && j < j1[r]) ? a[(int64_t)i * ld + j] : 0.0;
      }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = i0 + r * stride, j = 32 * (p + q * T) + lane;
        if (i < iend && j >= j0 && j < j1[r]) a[(int64_t)i * ld + j] = v[r][q] - s[r] * xv[q];
      }
  }
}

// Dense solver for one problem, run by a team of T CTAs (T = 1: one CTA; dsm: up to 200 KB of
// shared memory per CTA).  The FP64 reductions are shared out: the scaling, the two triangular
// solves, the Hessenberg reduction (columns for its left, rows for its right updates), the
// inverse iterations and the back-transformations; the Cholesky factorisation and the QR run
// on rank 0 while the others wait at the team barrier.  Every rank takes the same decisions
// from the same data (values read after a barrier), so the ranks leave together.
__device__ void dense_geig(const EigProblem pb, double* dsm, Shared& sh, Team tm = Team{0, 1, nullptr}) {
  const int m = pb.m;
  const int t = threadIdx.x, nt = blockDim.x;
  __shared__ TeamCtl local_ctl;
  __shared__ int bar_ok;
  const int R = tm.r, T = tm.T;
  TeamCtl* ctl = T > 1 ? tm.ctl : &local_ctl;
  auto sync = [&]() -> bool { return team_sync(tm, ctl, &bar_ok); };
  // column pieces of 32 belong to rank (piece mod T); rows to the team's warps in turn
  auto own_col = [&](int j) { return ((j >> 5) % T) == R; };
  const int64_t mm = (int64_t)m * m;
  double* L = pb.work;
  double* A = L + mm;
  double* Hh = A + mm;
  double* W = Hh + mm;            // 2 m^2: QR working copy, then Householder vectors as rows
  double* dsc = W + 2 * mm;
  double* hbeta = dsc + m;
  double* wr = hbeta + m;
  double* wi = wr + m;
  // each rank's two work vectors (m each) at the end of its shared memory (the left update's
  // partial sums fill the rest of it; the QR windows and the eigenvector buffers reuse it later)
  double* col = dsm + kEigSmemDoubles - 2 * (int64_t)m;
  double* vtmp = col + m;
  // per-warp inverse iteration: packed U, pivots; then the Hessenberg-basis eigenvectors
  double* Uw = pb.work + eig_base_doubles(m);                 // kVecSlots x m (m + 1)
  double* plw = Uw + (int64_t)kVecSlots * m * (m + 1);        // kVecSlots x 2m
  int* psw = reinterpret_cast<int*>(plw + (int64_t)kVecSlots * 2 * m);   // kVecSlots x m ints
  double* cvec = plw + (int64_t)kVecSlots * 3 * m;            // kMaxKeep x 2m

#ifdef BLM_EIG_TIMING
  long long tmark[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  long long hsub[6] = {0, 0, 0, 0, 0, 0}, hc = 0;   // Hessenberg: reflector, left, barrier, right, barrier
#define HS_T0() (hc = clock64())
#define HS_T(i) (hsub[i] += clock64() - hc, hc = clock64())
#else
#define HS_T0() ((void)0)
#define HS_T(i) ((void)0)
#endif
  EIG_MARK(0);
  if (t == 0) {
    sh.iscal[1] = ST_OK;
    sh.iscal[4] = 0;
    if (T == 1) {
      local_ctl.flag = ST_OK;
      local_ctl.qr_ok = 0;
      local_ctl.vec_fail = 0;
      local_ctl.anorm_bits = 0ull;
    }
  }
  __syncthreads();
  const int rw = t >> 5, rl = t & 31, rnw = nt >> 5;
  const int gw = R * rnw + rw, gnw = T * rnw;
  // shared memory: the per-warp inverse-iteration buffers (6 m) bound the dimension
  if (6 * (int64_t)m > kEigSmemDoubles) {
    if (t == 0) *pb.status = ST_NOCONV;
    return;
  }   // this warp among the team's warps
  auto own_row = [&](int i) { return (i % gnw) / rnw == R; };
  // the team's status word: any rank may set it; read after a barrier
  auto flag = [&]() { return *(volatile int*)&ctl->flag; };
  auto fail = [&](int code) {
    if (t == 0) *pb.status = code;
  };
  // ---- 1. scaling ----
  // (every rank needs all of dsc: each computes it into shared memory, rank 0 keeps the copy
  // the back-transformation reads).  S and H are read past L1 and the read-only cache: the
  // Davidson iteration writes its projected problem in the same kernel just before the solve.
  double* dscs = dsm;
  for (int i = t; i < m; i += nt) {
    const double s = __ldcg(pb.S + (int64_t)i * m + i);
    if (!(s > 0.0) || !isfinite(s)) ctl->flag = ST_NOT_PD;
    const double d = (s > 0.0) ? 1.0 / sqrt(s) : 0.0;
    dscs[i] = d;
    if (R == 0) dsc[i] = d;
  }
  __syncthreads();
  // (rows over the team's warps, columns over lanes: coalesced, no index division)
  for (int i = gw; i < m; i += gnw) {
    const double di = dscs[i];
    for (int j = rl; j < m; j += 32) {
      const int64_t idx = (int64_t)i * m + j;
      const double sv = __ldcg(pb.S + idx) * di * dscs[j];
      const double hv = __ldcg(pb.H + idx) * di * dscs[j];
      if (!isfinite(sv) || !isfinite(hv)) ctl->flag = ST_NONFINITE;
      L[idx] = sv;
      A[idx] = hv;
    }
  }
  if (!sync()) return fail(ST_NOCONV);
  if (flag() != ST_OK) return fail(flag());
  EIG_MARK(1);
  // The Davidson projection's overlap is the identity (S-orthonormal basis): L = I and A = H
  // as assembled above, so the Cholesky factorisation and the reduction are skipped.
  if (!(pb.flags & kEigUnitS)) {
    // ---- 2a. Cholesky (right-looking, lower), rows shared out ----
    // Step k reads column k below the diagonal and the pivot; the owners of its rows write the
    // factor's column k into row k of the upper triangle (unused: S is symmetric and only its
    // lower half is read) and update their trailing rows; the pivots' square roots go to hbeta
    // (free until the Hessenberg reduction).  Nothing read in a step is written in it, so one
    // team barrier per step suffices; the factor moves to the lower triangle at the end.
    for (int k = 0; k < m; ++k) {
      if (t == 0) {
        const double p = L[(int64_t)k * m + k];
        if (!(p > 1e-15)) {
          sh.iscal[1] = ST_NOT_PD;
        } else {
          sh.scal[0] = 1.0 / sqrt(p);
          if (R == 0) hbeta[k] = sqrt(p);
        }
      }
      __syncthreads();
      if (sh.iscal[1] != ST_OK) break;
      const double inv = sh.scal[0];
      for (int i = k + 1 + t; i < m; i += nt) {
        const double v = L[(int64_t)i * m + k] * inv;
        col[i] = v;
        if (own_row(i)) L[(int64_t)k * m + i] = v;
      }
      __syncthreads();
      const int i0 = k + 1 + ((gw - (k + 1)) % gnw + gnw) % gnw;   // first own row > k
      if (m <= kRows4Min) {
        for (int i = i0; i < m; i += gnw) row_axpy(L + (int64_t)i * m, col, col[i], k + 1, i + 1, rl);
      } else {
        for (int i = i0; i < m; i += 4 * gnw) {
          double sv[4];
          int j1[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int ir = i + r * gnw;
            sv[r] = ir < m ? col[ir] : 0.0;
            j1[r] = ir + 1;
          }
          rows4_axpy(L, m, i, gnw, m, sv, j1, col, k + 1, rl);
        }
      }
      if (!sync()) return fail(ST_NOCONV);
    }
    if (sh.iscal[1] == ST_OK) {
      // the factor into the lower triangle: row i <- column i of the upper triangle, pivot
      for (int i = gw; i < m; i += gnw) {
        for (int j = rl; j < i; j += 32) L[(int64_t)i * m + j] = L[(int64_t)j * m + i];
        if (rl == 0) L[(int64_t)i * m + i] = hbeta[i];
      }
    }
    if (R == 0 && t == 0 && sh.iscal[1] != ST_OK) ctl->flag = sh.iscal[1];
    if (!sync()) return fail(ST_NOCONV);
    if (flag() != ST_OK) return fail(flag());
    // ---- 2b. A <- L^-1 A (row forward substitution; columns are independent: each rank
    // takes its column pieces) ----
    for (int k = 0; k < m; ++k) {
      const double inv = 1.0 / L[(int64_t)k * m + k];
      for (int j = t; j < m; j += nt) {
        if (!own_col(j)) continue;
        const double v = A[(int64_t)k * m + j] * inv;
        A[(int64_t)k * m + j] = v;
        col[j] = v;
      }
      __syncthreads();
      if (m <= kRows4Min) {
        for (int i = k + 1 + rw; i < m; i += rnw)
          row_axpy_own(A + (int64_t)i * m, col, L[(int64_t)i * m + k], 0, m, rl, R, T);
      } else {
        for (int i = k + 1 + rw; i < m; i += 4 * rnw) {
          double sv[4];
          int j1[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int ir = i + r * rnw;
            sv[r] = ir < m ? L[(int64_t)ir * m + k] : 0.0;
            j1[r] = m;
          }
          rows4_axpy_own(A, m, i, rnw, m, sv, j1, col, 0, rl, R, T);
        }
      }
      __syncthreads();
    }
    if (!sync()) return fail(ST_NOCONV);
    // ---- 2c. A <- A L^-T (column forward substitution; rows are independent: each rank
    // takes its rows) ----
    for (int k = 0; k < m; ++k) {
      const double inv = 1.0 / L[(int64_t)k * m + k];
      for (int i = t; i < m; i += nt) {
        vtmp[i] = L[(int64_t)i * m + k];            // column k of L, read once
        if (!own_row(i)) continue;
        const double v = A[(int64_t)i * m + k] * inv;
        A[(int64_t)i * m + k] = v;
        col[i] = v;
      }
      __syncthreads();
      if (m <= kRows4Min) {
        for (int i = gw; i < m; i += gnw) row_axpy(A + (int64_t)i * m, vtmp, col[i], k + 1, m, rl);
      } else {
        for (int i = gw; i < m; i += 4 * gnw) {
          double sv[4];
          int j1[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int ir = i + r * gnw;
            sv[r] = ir < m ? col[ir] : 0.0;
            j1[r] = m;
          }
          rows4_axpy(A, m, i, gnw, m, sv, j1, vtmp, k + 1, rl);
        }
      }
      __syncthreads();
    }
    if (!sync()) return fail(ST_NOCONV);
  }
  EIG_MARK(2);
  // ---- 3. Householder reduction to Hessenberg form ----
  // Every rank forms column k's reflector from the same data; the left update (a reduction
  // over rows) is shared out by column pieces, the right update (a reduction over columns) by
  // rows, with a team barrier after each.
  for (int k = 0; k < m - 2; ++k) {
    HS_T0();
    double part = 0.0;
    for (int i = k + 2 + t; i < m; i += nt) {
      const double v = A[(int64_t)i * m + k];
      part += v * v;
    }
    const double sigma = block_sum(part, sh.red);
    if (t == 0) {
      const double x0 = A[(int64_t)(k + 1) * m + k];
      if (sigma == 0.0) {
        sh.scal[1] = 0.0;
        sh.scal[2] = 1.0;
      } else {
        const double mu = sqrt(x0 * x0 + sigma);
        const double v0 = (x0 <= 0.0) ? (x0 - mu) : (-sigma / (x0 + mu));
        sh.scal[1] = 2.0 * v0 * v0 / (sigma + v0 * v0);
        sh.scal[2] = v0;
      }
    }
    __syncthreads();
    const double beta = sh.scal[1], v0 = sh.scal[2];
    if (t == 0 && R == 0) hbeta[k] = beta;
    // u = (1, x[1:]/v0) into col[k+1..m-1]
    const double rv0 = rcp_nr(v0);
    for (int i = k + 1 + t; i < m; i += nt) col[i] = (i == k + 1) ? 1.0 : A[(int64_t)i * m + k] * rv0;
    __syncthreads();
    HS_T(0);
    if (beta != 0.0) {
      // left: rows k+1.., this rank's columns k..: w = beta u^T A from per-warp partial sums
      // over rows (each warp a slice of the rows, lanes over columns: coalesced, loads
      // independent), then A -= u w
      // (in chunks of columns that fit the shared memory before col and vtmp)
      double* wpart = dsm;                          // rnw x chunk
      const int chunk = max(32, (int)((kEigSmemDoubles - 2 * (int64_t)m) / rnw) / 32 * 32);
      for (int jb = (k >> 5) << 5; jb < m; jb += chunk) {
        const int je = min(m, jb + chunk);
        for (int p = first_piece(max(k, jb), R, T); 32 * p < je; p += T) {
          const int j = 32 * p + rl;
          if (j >= k && j < je) {
            const double* __restrict__ aj = A + j;
            const double* __restrict__ u = col;
            double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0, acc3 = 0.0;
            int i = k + 1 + rw;
            for (; i + 3 * rnw < m; i += 4 * rnw) {   // four independent loads in flight
              acc0 = fma(u[i], aj[(int64_t)i * m], acc0);
              acc1 = fma(u[i + rnw], aj[(int64_t)(i + rnw) * m], acc1);
              acc2 = fma(u[i + 2 * rnw], aj[(int64_t)(i + 2 * rnw) * m], acc2);
              acc3 = fma(u[i + 3 * rnw], aj[(int64_t)(i + 3 * rnw) * m], acc3);
            }
            for (; i < m; i += rnw) acc0 = fma(u[i], aj[(int64_t)i * m], acc0);
            wpart[rw * chunk + (j - jb)] = (acc0 + acc1) + (acc2 + acc3);
          }
        }
        __syncthreads();
        for (int j = max(k, jb) + t; j < je; j += nt) {
          if (!own_col(j)) continue;
          double sum = 0.0;
          for (int w2 = 0; w2 < rnw; ++w2) sum += wpart[w2 * chunk + (j - jb)];
          vtmp[j] = beta * sum;
        }
        __syncthreads();
      }
      if (m <= kRows4Min) {
        for (int i = k + 1 + rw; i < m; i += rnw)
          row_axpy_own(A + (int64_t)i * m, vtmp, col[i], k, m, rl, R, T);
      } else {
        for (int i = k + 1 + rw; i < m; i += 4 * rnw) {
          double sv[4];
          int j1[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int ir = i + r * rnw;
            sv[r] = ir < m ? col[ir] : 0.0;
            j1[r] = m;
          }
          rows4_axpy_own(A, m, i, rnw, m, sv, j1, vtmp, k, rl, R, T);
        }
      }
#ifdef BLM_EIG_TIMING
      __syncthreads();
#endif
      HS_T(1);
      if (!sync()) return fail(ST_NOCONV);
      HS_T(2);
      // right: this rank's rows, columns k+1..
      if (m <= kRows4Min) {
        for (int i = gw; i < m; i += gnw) {
          double zi = row_dot(A + (int64_t)i * m, col, k + 1, m, rl);
          for (int o = 16; o > 0; o >>= 1) zi += __shfl_xor_sync(0xffffffffu, zi, o);
          row_axpy(A + (int64_t)i * m, col, zi * beta, k + 1, m, rl);
        }
      } else {
        for (int i = gw; i < m; i += 4 * gnw) rows4_dot_axpy(A, m, i, gnw, m, col, beta, k + 1, m, rl);
      }
#ifdef BLM_EIG_TIMING
      __syncthreads();
#endif
      HS_T(3);
    }
    // store the reflector below the subdiagonal (the rank that updated column k)
    if (own_col(k))
      for (int i = k + 2 + t; i < m; i += nt) A[(int64_t)i * m + k] = col[i];
    if (!sync()) return fail(ST_NOCONV);
    HS_T(4);
  }
  // ---- Hessenberg copies: Hh (inverse iteration) and the QR working copy in W ----
  double amx = 0.0;
  for (int i = gw; i < m; i += gnw)
    for (int j = rl; j < m; j += 32) {
      const int64_t idx = (int64_t)i * m + j;
      const double v = (j >= i - 1) ? A[idx] : 0.0;
      Hh[idx] = v;
      amx = fmax(amx, fabs(v));
    }
  amx = block_max(amx, sh.red);
  if (t == 0) atomicMax(&ctl->anorm_bits, (unsigned long long)__double_as_longlong(amx));
  if (!sync()) return fail(ST_NOCONV);
  const double anorm =
      fmax(__longlong_as_double((long long)*(volatile unsigned long long*)&ctl->anorm_bits), 1e-300);
  // the QR runs on the matrix scaled by a power of two to max |entry| in [1/2, 1)
  int gex;
  frexp(anorm, &gex);
  const double gscale = ldexp(1.0, -gex);
  const int want = pb.mode == 1 ? 1 : pb.k;
  EIG_MARK(3);
  // ---- 4. all eigenvalues, the selection of the lowest, and their eigenvectors ----
  // With kEigLocate32 an FP32 QR only locates the eigenvalues: every kept one is recomputed in
  // FP64 by inverse iteration (its Rayleigh quotient; a second round shifted to that quotient
  // when the first leaves a residual above 1e-12 anorm), and the location is kept only if every
  // kept vector converged to 1e-12 anorm, no FP64 value moved by more than 1e-4 anorm from its
  // FP32 value, the kept eigenvalues lie below the lowest one left out by more than
  // max(10 x the largest such move, 1e-5 anorm), no two kept entries converged to one
  // eigenvector, and every kept complex pair keeps its imaginary part in FP64.  The output is
  // then ordered by the FP64 values.  Otherwise (and without the flag) the double-word QR
  // locates them (the FP64 QR if that fails) and the selection is redone.
  bool use32 = (pb.flags & kEigLocate32) != 0;
  int nsel = 0, njob = 0;
  const int warp = t >> 5, lane = t & 31;
  for (;;) {
    // the QR on rank 0; qr_ok: 1 located in FP32, 2 in double words (or FP64), 0 failed
    if (R == 0) {
    bool ok = false;
    int how = 0;
    if (use32) {
      float* Wf = reinterpret_cast<float*>(W);
      for (int64_t idx = t; idx < mm; idx += nt) Wf[idx] = (float)(Hh[idx] * gscale);
      if (t == 0) sh.iscal[5] = 1;
      __syncthreads();
      ok = hqr_windowed<float>(Wf, m, wr, wi, anorm * gscale, dsm, sh);
      __syncthreads();
      for (int i = t; i < m; i += nt)
        if (!isfinite(wr[i]) || !isfinite(wi[i])) sh.iscal[5] = 0;
      __syncthreads();
      if (ok && sh.iscal[5] != 0) how = 1;
    }
    if (how == 0) {
      dw* Wd = reinterpret_cast<dw*>(W);
      for (int64_t idx = t; idx < mm; idx += nt) Wd[idx] = dw_of_double(Hh[idx] * gscale);
      if (t == 0) sh.iscal[5] = 1;
      __syncthreads();
      ok = hqr_windowed<dw>(Wd, m, wr, wi, anorm * gscale, dsm, sh);
      __syncthreads();
      for (int i = t; i < m; i += nt)
        if (!isfinite(wr[i]) || !isfinite(wi[i])) sh.iscal[5] = 0;
      __syncthreads();
      if (!ok || sh.iscal[5] == 0) {
#ifdef BLM_EIG_DEBUG
        if (t == 0) printf("eig: problem %d double-word QR failed, FP64 QR\n", (int)blockIdx.x);
#endif
        for (int64_t idx = t; idx < mm; idx += nt) W[idx] = Hh[idx] * gscale;
        __syncthreads();
        ok = hqr_windowed<double>(W, m, wr, wi, anorm * gscale, dsm, sh);
        __syncthreads();
      }
      if (ok) how = 2;
    }
    if (how != 0)
      for (int i = t; i < m; i += nt) {
        wr[i] /= gscale;
        wi[i] /= gscale;
      }
    __syncthreads();
    if (t == 0) ctl->qr_ok = how;
    }
    if (!sync()) return fail(ST_NOCONV);
    {
      const int how = *(volatile int*)&ctl->qr_ok;
      if (how == 0) return fail(ST_NOCONV);
      use32 = how == 1;
    }
    // ---- selection of the lowest real parts; eigenvector jobs ----
    // A job is one complex pair (both of its parts) or a run of selected real eigenvalues closer
    // to each other than 1e-9 anorm (a numerically repeated eigenvalue): one warp computes the
    // run's vectors one after another, each orthogonalised against the earlier ones.  (FP32
    // locations are not grouped: kept eigenvalues that close fail the check below.)
    if (t == 0) {
      int ns = 0;
      for (int i = 0; i < m; ++i) vtmp[i] = 0.0;   // used flags
      while (ns < want) {
        int best = -1;
        double bv = 0.0;
        for (int i = 0; i < m; ++i) {
          if (vtmp[i] != 0.0) continue;
          if (best < 0 || wr[i] < bv) {
            best = i;
            bv = wr[i];
          }
        }
        if (best < 0) break;
        vtmp[best] = 1.0;
        if (wi[best] != 0.0) {
          // the conjugate partner is adjacent (same 2 x 2 block)
          int partner = -1;
          if (best + 1 < m && wi[best + 1] == -wi[best] && wr[best + 1] == wr[best]) partner = best + 1;
          if (best > 0 && wi[best - 1] == -wi[best] && wr[best - 1] == wr[best]) partner = best - 1;
          if (partner >= 0) vtmp[partner] = 1.0;
          const int pos = wi[best] > 0.0 ? best : (partner >= 0 ? partner : best);
          sh.sel_idx[ns] = pos;
          sh.sel_part[ns] = 1;
          ++ns;
          if (ns < want) {
            sh.sel_idx[ns] = pos;
            sh.sel_part[ns] = 2;
            ++ns;
          }
        } else {
          sh.sel_idx[ns] = best;
          sh.sel_part[ns] = 0;
          ++ns;
        }
      }
      double lo_out = INFINITY;   // the lowest real part left out
      for (int i = 0; i < m; ++i)
        if (vtmp[i] == 0.0 && wr[i] < lo_out) lo_out = wr[i];
      sh.scal[3] = lo_out;
      const double run_gap = use32 ? 0.0 : 1e-9 * anorm;
      int nj = 0;
      for (int q = 0; q < ns;) {
        int len = 1;
        if (sh.sel_part[q] == 1) {
          len = (q + 1 < ns && sh.sel_part[q + 1] == 2) ? 2 : 1;
        } else {
          while (q + len < ns && sh.sel_part[q + len] == 0 &&
                 wr[sh.sel_idx[q + len]] - wr[sh.sel_idx[q + len - 1]] <= run_gap)
            ++len;
        }
        sh.job_q0[nj] = q;
        sh.job_len[nj] = len;
        ++nj;
        q += len;
      }
      sh.iscal[2] = ns;
      sh.iscal[3] = nj;
      for (int q = 0; q < ns; ++q) sh.out_pos[q] = q;
      if (pb.mode == 1 && ns > 0 && sh.sel_part[0] != 0 && !use32) sh.iscal[1] = ST_COMPLEX;
    }
    __syncthreads();
    if (sh.iscal[1] != ST_OK) {
      if (t == 0) *pb.status = sh.iscal[1];
      return;
    }
    nsel = sh.iscal[2];
    njob = sh.iscal[3];
    EIG_MARK(4);
    // ---- 5. eigenvectors of the Hessenberg matrix: inverse iteration, one warp per job ----
    // The shift is the located eigenvalue, so three solves from a fixed start vector converge;
    // the residual ||Hh y - lambda y|| is checked before the vector is used.
    // (the team's vector warps share the kVecSlots factor slots: global vector warp gv)
    const int nvw = min(min(kVecWarps, max(1, kVecSlots / T)), (int)((kEigSmemDoubles) / (6 * (int64_t)m)));
    const int gv = R * nvw + warp, gnv = T * nvw;
    if (warp < nvw) {
      double* cur = dsm + (int64_t)warp * 6 * m;
      double* nxt = cur + 2 * m;
      double* yv = nxt + 2 * m;
      double* U = Uw + (int64_t)gv * m * (m + 1);
      double* pl = plw + (int64_t)gv * 2 * m;
      int* ps = psw + (int64_t)gv * m;
      const double pert = anorm * 1e-14;   // keeps the factorisation nonsingular at an eigenvalue
      for (int j = gv; j < njob; j += gnv) {
        const int q0 = sh.job_q0[j], len = sh.job_len[j];
        const bool cx = sh.sel_part[q0] != 0;
        double sprev = NAN;
        for (int c = 0; c < len; ++c) {
          const int idx = sh.sel_idx[q0 + c];
          const double lre = wr[idx], lim = cx ? wi[idx] : 0.0;
          // An FP32 location gets a second round, shifted to the first round's Rayleigh
          // quotient, when the first leaves a residual above 1e-12 anorm (a neighbour closer
          // than the FP32 error allows slows the first round's convergence).
          double sre = lre, sim = lim, qre = 0.0, qim = 0.0, res = INFINITY;
          const int rounds = use32 ? 2 : 1;
          for (int round = 0; round < rounds; ++round) {
            if (round == 1) {
              if (res <= 1e-12 * anorm) break;
              sre = qre;
              sim = cx ? qim : 0.0;
              sprev = NAN;
            }
            if (cx) {
              warp_hess_lu<true>(Hh, m, sre + pert, sim, pert, cur, nxt, U, pl, ps);
            } else if (!(sre == sprev)) {
              warp_hess_lu<false>(Hh, m, sre + pert, 0.0, pert, cur, nxt, U, pl, ps);
              sprev = sre;
            }
            if (round == 0) {
              for (int i = lane; i < m; i += 32) {
                yv[i] = 1.0 + 0.1 * (double)(((i + 31 * c) * 7919) % 97) / 97.0;
                yv[m + i] = 0.0;
              }
              __syncwarp();
            }
            for (int it = 0; it < (round == 0 ? 3 : 2); ++it) {
              if (cx) {
                warp_hess_solve<true>(m, pert, U, pl, ps, yv);
              } else {
                warp_hess_solve<false>(m, pert, U, pl, ps, yv);
                // orthogonalise against the run's earlier vectors (unit norm, stored in cvec)
                for (int e = 0; e < c; ++e) {
                  const double* ve = cvec + (int64_t)(q0 + e) * 2 * m;
                  const double d = warp_dot(ve, yv, m);
                  for (int i = lane; i < m; i += 32) yv[i] -= d * ve[i];
                  __syncwarp();
                }
              }
            }
            // normalise; H y into cur (re | im); the Rayleigh quotient y^H H y / y^H y becomes
            // the eigenvalue (FP64 accurate whatever the QR's precision); then the residual
            double nrm = 0.0;
            for (int i = lane; i < m; i += 32) nrm += yv[i] * yv[i] + (cx ? yv[m + i] * yv[m + i] : 0.0);
            nrm = sqrt(warp_sum(nrm));
            const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
            for (int i = lane; i < 2 * m; i += 32) yv[i] = (i < m || cx) ? yv[i] * inv : 0.0;
            __syncwarp();
            for (int i = 0; i < m; ++i) {
              const double* hrow = Hh + (int64_t)i * m;
              double hr = 0.0, hm = 0.0;
              for (int k2 = (i > 0 ? i - 1 : 0) + lane; k2 < m; k2 += 32) {
                hr = fma(hrow[k2], yv[k2], hr);
                if (cx) hm = fma(hrow[k2], yv[m + k2], hm);
              }
              hr = warp_sum(hr);
              if (cx) hm = warp_sum(hm);
              if (lane == 0) {
                cur[i] = hr;
                cur[m + i] = hm;
              }
            }
            __syncwarp();
            qre = 0.0;
            qim = 0.0;
            for (int i = lane; i < m; i += 32) {
              qre += yv[i] * cur[i] + (cx ? yv[m + i] * cur[m + i] : 0.0);
              if (cx) qim += yv[i] * cur[m + i] - yv[m + i] * cur[i];
            }
            qre = warp_sum(qre);   // y is unit: y^H y = 1
            qim = cx ? warp_sum(qim) : 0.0;
            double rr = 0.0;
            for (int i = lane; i < m; i += 32) {
              const double er = cur[i] - (qre * yv[i] - qim * yv[m + i]);
              const double ei = cx ? cur[m + i] - (qre * yv[m + i] + qim * yv[i]) : 0.0;
              rr += er * er + ei * ei;
            }
            res = sqrt(warp_sum(rr));
          }
          if (lane == 0) {
            const bool conv = res <= (use32 ? 1e-12 : 1e-9) * anorm;
            if (use32) {
              // an FP32 location must give a converged vector whose quotient stays near it
              const double mv = fabs(qre - lre);
              const double e = (conv && mv <= 1e-4 * anorm) ? mv : INFINITY;
              ctl->sel_err[q0 + c] = e;
              ctl->sel_qim[q0 + c] = qim;
              if (cx && c == 0 && len == 2) {
                ctl->sel_err[q0 + 1] = e;
                ctl->sel_qim[q0 + 1] = qim;
              }
              if (e != INFINITY) wr[idx] = qre;
            } else {
              // A converged vector (residual <= 1e-9 ||H||, quotient next to the QR value) gives
              // the eigenvalue as its Rayleigh quotient; otherwise the QR value stands (a nearly
              // defective eigenvalue converges slowly under inverse iteration).  Only a vector
              // that is no eigenvector at all (residual above 1e-6 ||H||) fails the solve.
              if (!(res <= 1e-6 * anorm)) ctl->vec_fail = 1;
              if (conv && fabs(qre - lre) <= 1e-6 * anorm) wr[idx] = qre;
            }
#ifdef BLM_EIG_DEBUG
            if (!conv || !(fabs(qre - lre) <= 1e-6 * anorm))
              printf("eig: problem %d eigenvector %d residual %.3e shift %.15g quotient %.15g (anorm %.3e)%s\n",
                     (int)blockIdx.x, q0 + c, res, lre, qre, anorm, use32 ? " [fp32 location]" : "");
#endif
          }
          double* dst = cvec + (int64_t)(q0 + c) * 2 * m;
          for (int i = lane; i < 2 * m; i += 32) dst[i] = yv[i];
          if (cx && c == 0 && len == 2) {
            double* dst2 = cvec + (int64_t)(q0 + 1) * 2 * m;
            for (int i = lane; i < 2 * m; i += 32) dst2[i] = yv[i];
          }
          __syncwarp();
          if (cx) break;   // the pair's second entry shares the vector
        }
      }
    }
    if (!sync()) return fail(ST_NOCONV);
    if (!use32) break;
    // ---- is the FP32 location good enough? (every rank decides alike) ----
    if (t == 0) {
      double mv = 0.0, top = -INFINITY;
      for (int q = 0; q < nsel; ++q) {
        mv = fmax(mv, *(volatile double*)&ctl->sel_err[q]);   // INFINITY for a failed vector
        top = fmax(top, wr[sh.sel_idx[q]]);
      }
      const double sep = fmax(10.0 * mv, 1e-5 * anorm);
      // membership: the kept eigenvalues must lie clearly below the first one left out
      bool good = mv <= 1e-4 * anorm && !(sh.scal[3] - top <= sep);
      for (int q = 0; q < nsel && good; ++q) {
        const int iq = sh.sel_idx[q];
        // a pair must stay a pair: the FP64 quotient's imaginary part agrees with the FP32 one
        // (two close real eigenvalues located as a pair give a real quotient)
        if (sh.sel_part[q] != 0) {
          const double qi = *(volatile double*)&ctl->sel_qim[q];
          if (!(fabs(qi) > 10.0 * fabs(qi - wi[iq]) && fabs(qi) > 1e-9 * anorm)) good = false;
        }
        if (pb.mode == 1 && q == 0 && sh.sel_part[q] != 0) good = false;   // must be real
        // two kept entries whose vectors converged to one eigenvector
        for (int r = q + 1; r < nsel && good; ++r) {
          const int ir = sh.sel_idx[r];
          if (ir != iq && fabs(wr[ir] - wr[iq]) <= 1e-9 * anorm) good = false;
        }
      }
      // a pair cut by N_K (its real part kept alone) must stay the highest kept eigenvalue
      if (good && nsel > 0 && sh.sel_part[nsel - 1] == 1) {
        const double vp = wr[sh.sel_idx[nsel - 1]];
        for (int q = 0; q < nsel - 1 && good; ++q)
          if (sh.sel_idx[q] != sh.sel_idx[nsel - 1] && !(wr[sh.sel_idx[q]] < vp - sep)) good = false;
      }
      // output in ascending order of the FP64 values (a pair's two entries stay together)
      if (good) {
        int pos = 0;
        bool placed[kMaxKeep];
        for (int q = 0; q < nsel; ++q) placed[q] = false;
        for (;;) {
          int bq = -1;
          for (int q = 0; q < nsel; ++q) {
            if (placed[q] || sh.sel_part[q] == 2) continue;
            if (bq < 0 || wr[sh.sel_idx[q]] < wr[sh.sel_idx[bq]]) bq = q;
          }
          if (bq < 0) break;
          placed[bq] = true;
          sh.out_pos[bq] = pos++;
          if (sh.sel_part[bq] == 1 && bq + 1 < nsel && sh.sel_part[bq + 1] == 2) {
            placed[bq + 1] = true;
            sh.out_pos[bq + 1] = pos++;
          }
        }
      }
      sh.iscal[6] = good ? 1 : 0;
#ifdef BLM_EIG_DEBUG
      if (!good && R == 0)
        printf("eig: problem %d (m %d) FP32 location rejected: max move %.3e, gap to the first left "
               "out %.3e, separation needed %.3e (anorm %.3e); kept:\n",
               (int)blockIdx.x, m, mv, sh.scal[3] - top, sep, anorm);
      if (!good && R == 0)
        for (int q = 0; q < nsel; ++q)
          printf("  entry %d idx %d part %d re %.15g im %.3e err %.3e\n", q, sh.sel_idx[q],
                 sh.sel_part[q], wr[sh.sel_idx[q]], wi[sh.sel_idx[q]], ctl->sel_err[q]);
#endif
    }
    __syncthreads();
    if (sh.iscal[6]) break;
    use32 = false;   // locate again with double words
    if (!sync()) return fail(ST_NOCONV);   // (every rank has read wr before the QR rewrites it)
  }
  // Householder vectors as rows for coalesced per-warp back-transformation (W is free now)
  for (int k = gw; k < m; k += gnw)
    for (int i = rl; i < m; i += 32)
      W[(int64_t)k * m + i] = (i >= k + 2 && k < m - 2) ? A[(int64_t)i * m + k] : 0.0;
  if (!sync()) return fail(ST_NOCONV);
  if (*(volatile int*)&ctl->vec_fail != 0) return fail(ST_NOCONV);
  EIG_MARK(5);
  // ---- 6. back-transformation v = D L^-T Q y, one warp per selected direction ----
  // A complex eigenvector is rotated so that its largest-magnitude component is real and
  // positive; its real part (kept alone when N_K ends inside the pair) is then well defined.
  const int nw = min(nt >> 5, (int)(kEigSmemDoubles / (2 * (int64_t)m)));
  for (int q = R * nw + warp; q < nsel && warp < nw; q += T * nw) {
    const int part = sh.sel_part[q];
    double* vr2 = dsm + (int64_t)warp * 2 * m;
    double* vi2 = vr2 + m;
    const double* src = cvec + (int64_t)q * 2 * m;
    for (int i = lane; i < m; i += 32) {
      vr2[i] = src[i];
      vi2[i] = src[m + i];
    }
    __syncwarp();
    warp_back_transform(W, hbeta, L, dsc, m, vr2);
    if (part) {
      warp_back_transform(W, hbeta, L, dsc, m, vi2);
      double bv = -1.0;
      int best = 0;
      for (int i = lane; i < m; i += 32) {
        const double a2 = vr2[i] * vr2[i] + vi2[i] * vi2[i];
        if (a2 > bv) {
          bv = a2;
          best = i;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, best, o);
        if (ob > bv || (ob == bv && oi < best)) {
          bv = ob;
          best = oi;
        }
      }
      const double nr = sqrt(bv);
      const double cc = vr2[best] / nr, ss = vi2[best] / nr;
      __syncwarp();
      for (int i = lane; i < m; i += 32) {
        const double a2 = vr2[i], b2 = vi2[i];
        vr2[i] = a2 * cc + b2 * ss;       // (a + i b)(c - i s)
        vi2[i] = b2 * cc - a2 * ss;
      }
      __syncwarp();
    }
    const int op = sh.out_pos[q];
    double* out = pb.vec + (int64_t)op * m;
    const double* res = (part == 2) ? vi2 : vr2;
    for (int i = lane; i < m; i += 32) out[i] = res[i];
    if (lane == 0) pb.lam[op] = wr[sh.sel_idx[q]];
    __syncwarp();
  }
  if (!sync()) return fail(ST_NOCONV);
  if (t == 0 && R == 0) *pb.status = (nsel == (pb.mode == 1 ? 1 : pb.k)) ? ST_OK : ST_NOCONV;
  EIG_MARK(6);
#ifdef BLM_EIG_TIMING
  if (t == 0 && R == 0 && blockIdx.x == 0)
    printf("eig timing m=%d: scale %lld chol+std %lld hess %lld qr %lld vec %lld back %lld cycles; "
           "hessenberg: reflector %lld left %lld barrier %lld right %lld store+barrier %lld\n",
           m, tmark[1] - tmark[0], tmark[2] - tmark[1], tmark[3] - tmark[2], tmark[4] - tmark[3],
           tmark[5] - tmark[4], tmark[6] - tmark[5], hsub[0], hsub[1], hsub[2], hsub[3], hsub[4]);
#endif
}

__global__ void __launch_bounds__(kEigThreads)
eig_kernel(const EigProblem* __restrict__ probs) {
  extern __shared__ double dsm[];
  __shared__ Shared sh;
  const EigProblem pb = probs[blockIdx.x];
  if (pb.run_if_noconv && *pb.run_if_noconv != ST_NOCONV) return;
  dense_geig(pb, dsm, sh);
}

// CTA c of a team launch solves problem prob[c] as rank rank[c] of size[c] CTAs.
// A team launch: CTA c < nteam solves problem prob[c] as rank rank[c] of size[c] CTAs; then
// every CTA takes the problems of the queue (largest first) one at a time from a shared counter.
constexpr int kTeamGridMax = 160;
constexpr int kQueueMax = 4096;
struct TeamMap {
  uint16_t prob[kTeamGridMax];
  uint8_t rank[kTeamGridMax];
  uint8_t size[kTeamGridMax];
  int nteam, nqueue;
  uint16_t queue[kQueueMax];
};

template <bool kQueue>
__global__ void __launch_bounds__(kEigThreads, 1)
eig_team_kernel(const EigProblem* __restrict__ probs, TeamCtl* ctl, int* queue_head,
                const __grid_constant__ TeamMap map) {
  extern __shared__ double dsm[];
  __shared__ Shared sh;
  if constexpr (!kQueue) {
    // one task per CTA (fewer problems than SMs)
    const int p = map.prob[blockIdx.x];
    const EigProblem pb = probs[p];
    if (pb.run_if_noconv && *pb.run_if_noconv != ST_NOCONV) return;
    dense_geig(pb, dsm, sh, Team{(int)map.rank[blockIdx.x], (int)map.size[blockIdx.x], ctl + p});
  } else {
  __shared__ int qi;
  bool first = true;
  for (;;) {
    // (one call site of the solver, so that it is inlined)
    int p;
    Team tm{0, 1, nullptr};
    if (first && (int)blockIdx.x < map.nteam) {
      p = map.prob[blockIdx.x];
      tm = Team{(int)map.rank[blockIdx.x], (int)map.size[blockIdx.x], ctl + p};
    } else {
      __syncthreads();   // (every thread is done with the previous problem and with qi)
      if (threadIdx.x == 0) qi = map.nqueue > 0 ? atomicAdd(queue_head, 1) : map.nqueue;
      __syncthreads();
      if (qi >= map.nqueue) break;
      p = map.queue[qi];
    }
    first = false;
    const EigProblem pb = probs[p];
    if (pb.run_if_noconv && *pb.run_if_noconv != ST_NOCONV) continue;
    dense_geig(pb, dsm, sh, tm);
  }
  }
}

// ---------------------------------------------------------------------------------------------
// Generalized Davidson for the lowest eigenpair of H c = lambda S c (the combined problem of
// Eq. 7 when it is too large for the dense QR on one SM).  The basis V is kept S-orthonormal, so
// the projected problem V^T H V y = theta y is a small standard eigenproblem (solved with the
// dense routine above); the Ritz pair with the lowest real part is expanded with the diagonal
// preconditioner t = -(diag H - theta diag S)^-1 r, starting from the Psi direction e_0.
// Converged when ||H u - theta S u|| <= tol * ||S u|| * max(1, |theta|), or when that ratio has
// stayed within 10 tol for ten iterations without halving (the rounding floor).
// ---------------------------------------------------------------------------------------------
constexpr int kDavMax = 40;

__device__ double dotv(const double* a, const double* b, int m, Shared& sh) {
  double p = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) p = fma(a[i], b[i], p);
  return block_sum(p, sh.red);
}

// Control block of the grid-wide Davidson (global memory, zeroed before the launch).
struct DavCtl {
  unsigned int count;      // grid barrier: arrivals in the current generation
  unsigned int gen;        // grid barrier: generation
  int cmd;                 // 1: matrix-vector products of x, 0: done
  int err;                 // a barrier wait ran out
  const double* x;
};
constexpr uint32_t kGridSpinLimit = 1u << 24;

// Grid barrier of a cooperative launch (all CTAs resident), bounded: a wait that runs out sets
// err and returns false on every CTA that gives up.
__device__ bool grid_barrier(DavCtl* c, int* ok_smem) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = &c->gen;
    const unsigned int g = *vgen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(&c->count, 1u) == gridDim.x - 1) {
      atomicExch(&c->count, 0u);
      __threadfence();
      atomicAdd(&c->gen, 1u);
    } else {
      uint32_t i = 0;
      while (*vgen == g) {
        if (++i > kGridSpinLimit || *(volatile int*)&c->err) {
          ok = 0;
          atomicExch(&c->err, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    *ok_smem = ok;
  }
  __syncthreads();
  return *ok_smem != 0;
}

// This CTA's rows of y_H = H x and y_S = S x: global warp w takes rows w, w + all warps, ...;
// x is read past L1 (CTA 0 rewrites it between products).
__device__ void grid_rows_matvec(const double* __restrict__ H, const double* __restrict__ S, int m,
                                 const double* x, double* yH, double* yS) {
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int nw = gridDim.x * (blockDim.x >> 5);
  for (int i = gw; i < m; i += nw) {
    const double* __restrict__ hr = H + (int64_t)i * m;
    const double* __restrict__ sr = S + (int64_t)i * m;
    double h0 = 0.0, h1 = 0.0, s0 = 0.0, s1 = 0.0;
    int j = lane;
    for (; j + 32 < m; j += 64) {
      const double xa = __ldcg(x + j), xb = __ldcg(x + j + 32);
      h0 = fma(hr[j], xa, h0);
      s0 = fma(sr[j], xa, s0);
      h1 = fma(hr[j + 32], xb, h1);
      s1 = fma(sr[j + 32], xb, s1);
    }
    if (j < m) {
      const double xa = __ldcg(x + j);
      h0 = fma(hr[j], xa, h0);
      s0 = fma(sr[j], xa, s0);
    }
    double h = h0 + h1, sv = s0 + s1;
    for (int o = 16; o > 0; o >>= 1) {
      h += __shfl_xor_sync(0xffffffffu, h, o);
      sv += __shfl_xor_sync(0xffffffffu, sv, o);
    }
    if (lane == 0) {
      yH[i] = h;
      yS[i] = sv;
    }
  }
}

__global__ void __launch_bounds__(kEigThreads)
davidson_kernel(const EigProblem* __restrict__ probs, double tol, int max_iter, DavCtl* ctl) {
  extern __shared__ double dsm[];
  __shared__ Shared sh;
  __shared__ double hk[kDavMax * kDavMax];
  __shared__ double coef[kDavMax];
  __shared__ int bar_ok;
  const EigProblem pb = probs[0];
  const int m = pb.m;
  const int t = threadIdx.x, nt = blockDim.x;
  double* V = pb.work;                       // kDavMax x m
  double* HV = V + (int64_t)kDavMax * m;     // rows (H v_j)
  double* SV = HV + (int64_t)kDavMax * m;    // rows (S v_j)
  double* u = SV + (int64_t)kDavMax * m;
  double* Hu = u + m;
  double* Su = Hu + m;
  double* r = Su + m;
  double* dH = r + m;
  double* dS = dH + m;
  double* small = dS + m;                    // small problem: S (k^2) | H (k^2) | work | lam | vec
  const int ks = kDavMax;
  double* sS = small;
  double* sH = sS + ks * ks;
  double* sW = sH + ks * ks;
  double* sLam = sW + eig_total_doubles(ks);
  double* sVec = sLam + 2;
  int32_t* sStat = reinterpret_cast<int32_t*>(sVec + ks);
  double* yHs = sVec + ks + 2;               // matvec results of all CTAs (m each)
  double* ySs = yHs + m;

  // CTAs other than 0 only compute their rows of the matrix-vector products CTA 0 asks for
  if (blockIdx.x != 0) {
    for (;;) {
      if (!grid_barrier(ctl, &bar_ok)) return;                 // command posted
      if (((volatile DavCtl*)ctl)->cmd == 0) return;
      grid_rows_matvec(pb.H, pb.S, m, ((volatile DavCtl*)ctl)->x, yHs, ySs);
      if (!grid_barrier(ctl, &bar_ok)) return;                 // rows written
    }
  }
  // y_H = H x, y_S = S x over the whole grid, then copied (bypassing L1) into place
  auto grid_matvec = [&](const double* x, double* yH, double* yS) -> bool {
    if (t == 0) {
      ctl->x = x;
      ctl->cmd = 1;
      __threadfence();
    }
    if (!grid_barrier(ctl, &bar_ok)) return false;
    grid_rows_matvec(pb.H, pb.S, m, x, yHs, ySs);
    if (!grid_barrier(ctl, &bar_ok)) return false;
    for (int i = t; i < m; i += nt) {
      yH[i] = __ldcg(yHs + i);
      yS[i] = __ldcg(ySs + i);
    }
    __syncthreads();
    return true;
  };
  auto release = [&]() {
    if (t == 0) {
      ctl->cmd = 0;
      __threadfence();
    }
    grid_barrier(ctl, &bar_ok);
  };

  for (int i = t; i < m; i += nt) {
    dH[i] = pb.H[(int64_t)i * m + i];
    dS[i] = pb.S[(int64_t)i * m + i];
  }
  __syncthreads();
  if (!(dS[0] > 0.0)) {
    if (t == 0) *pb.status = ST_NOT_PD;
    release();
    return;
  }
  // v_0 = e_0 / sqrt(S_00)
  for (int i = t; i < m; i += nt) V[i] = (i == 0) ? 1.0 / sqrt(dS[0]) : 0.0;
  __syncthreads();
  if (!grid_matvec(V, HV, SV)) {
    if (t == 0) *pb.status = ST_NOCONV;
    return;
  }
  int k = 1;
  bool fresh = true;      // projected matrix must be rebuilt (start, restart)
  double theta = 0.0;
  int status = ST_NOCONV;
  double best_rel = INFINITY;
  int since_best = 0;
#ifdef BLM_EIG_TIMING
  long long dt[5] = {0, 0, 0, 0, 0}, dc0 = clock64();
  int dits = 0;
#define DAV_T(i) (dt[i] += clock64() - dc0, dc0 = clock64())
#else
#define DAV_T(i) ((void)0)
#endif
  for (int it = 0; it < max_iter; ++it) {
#ifdef BLM_EIG_TIMING
    dits = it + 1;
#endif
    // projected matrix: only the newest row and column change between restarts; one warp per
    // dot product, all of them between two barriers
    {
      const int np = fresh ? k * k : 2 * k - 1;
      const int lane = t & 31, wid = t >> 5, nw = nt >> 5;
      for (int q = wid; q < np; q += nw) {
        int i, j;
        if (fresh) {
          i = q / k;
          j = q - i * k;
        } else if (q < k) {
          i = k - 1;   // the new row
          j = q;
        } else {
          i = q - k;   // the new column, rows above the new row
          j = k - 1;
        }
        const double* vi = V + (int64_t)i * m;
        const double* hj = HV + (int64_t)j * m;
        double acc = 0.0;
        for (int e = lane; e < m; e += 32) acc = fma(vi[e], hj[e], acc);
        acc = warp_sum(acc);
        if (lane == 0) hk[i * kDavMax + j] = acc;
      }
    }
    __syncthreads();
    fresh = false;
    for (int q = t; q < k * k; q += nt) {
      const int i = q / k, j = q % k;
      sH[q] = hk[i * kDavMax + j];
      sS[q] = (i == j) ? 1.0 : 0.0;
    }
    if (t == 0) *sStat = ST_OK;
    __syncthreads();
    DAV_T(0);
    // (double-word location: the Ritz pair must be accurate to the Davidson tolerance)
    EigProblem sp{k, 1, 0, kEigUnitS, sS, sH, sW, sLam, sVec, sStat};
    dense_geig(sp, dsm, sh);
    __syncthreads();
    DAV_T(1);
    if (*sStat != ST_OK) {
      status = *sStat;
      break;
    }
    theta = sLam[0];
    // Ritz vector and its images
    for (int i = t; i < m; i += nt) {
      double a = 0.0, b = 0.0, c = 0.0;
      for (int j = 0; j < k; ++j) {
        const double y = sVec[j];
        a = fma(y, V[(int64_t)j * m + i], a);
        b = fma(y, HV[(int64_t)j * m + i], b);
        c = fma(y, SV[(int64_t)j * m + i], c);
      }
      u[i] = a;
      Hu[i] = b;
      Su[i] = c;
      r[i] = b - theta * c;
    }
    __syncthreads();
    const double rn = sqrt(dotv(r, r, m, sh));
    const double sn = sqrt(dotv(Su, Su, m, sh));
    DAV_T(2);
    // Converged at tol; or, where rounding keeps the residual from reaching tol (its floor is
    // about m eps ||H|| ||u||), once it has stayed within 10 tol for ten iterations without
    // halving.
    const double rel = rn / (sn * fmax(1.0, fabs(theta)));
    if (rel < 0.5 * best_rel) {
      best_rel = rel;
      since_best = 0;
    } else {
      ++since_best;
    }
    if (rel <= tol || (best_rel <= 10.0 * tol && since_best >= 10)) {
      status = ST_OK;
      break;
    }
    // restart: keep only the Ritz vector (S-normalised)
    if (k == kDavMax) {
      const double nu = sqrt(dotv(u, Su, m, sh));
      for (int i = t; i < m; i += nt) {
        V[i] = u[i] / nu;
        HV[i] = Hu[i] / nu;
        SV[i] = Su[i] / nu;
      }
      __syncthreads();
      k = 1;
      fresh = true;
    }
    // correction t = -r / (dH - theta dS), S-orthogonalised against V twice
    double* tv = V + (int64_t)k * m;
    for (int i = t; i < m; i += nt) {
      double den = dH[i] - theta * dS[i];
      if (fabs(den) < 1e-8 * fmax(1.0, fabs(dH[i]))) den = den < 0 ? -1e-8 : 1e-8;
      tv[i] = -r[i] / den;
    }
    __syncthreads();
    // classical Gram-Schmidt in the S inner product, twice: the k coefficients by one warp each,
    // then one combined update
    for (int pass = 0; pass < 2; ++pass) {
      const int lane = t & 31, wid = t >> 5, nw = nt >> 5;
      for (int j = wid; j < k; j += nw) {
        const double* sj = SV + (int64_t)j * m;
        double acc = 0.0;
        for (int e = lane; e < m; e += 32) acc = fma(sj[e], tv[e], acc);
        acc = warp_sum(acc);
        if (lane == 0) coef[j] = acc;
      }
      __syncthreads();
      for (int i = t; i < m; i += nt) {
        double x = tv[i];
        for (int j = 0; j < k; ++j) x -= coef[j] * V[(int64_t)j * m + i];
        tv[i] = x;
      }
      __syncthreads();
    }
    double* stv = SV + (int64_t)k * m;
    double* htv = HV + (int64_t)k * m;
    DAV_T(3);
    if (!grid_matvec(tv, htv, stv)) {
      if (t == 0) *pb.status = ST_NOCONV;
      return;
    }
    const double nn = dotv(tv, stv, m, sh);
    if (!(nn > 1e-300)) {
      status = ST_NOCONV;
      break;
    }
    const double inv = 1.0 / sqrt(nn);
    for (int i = t; i < m; i += nt) {
      tv[i] *= inv;
      stv[i] *= inv;
      htv[i] *= inv;
    }
    __syncthreads();
    DAV_T(4);
    ++k;
  }
#ifdef BLM_EIG_TIMING
  if (t == 0)
    printf("davidson m=%d iterations %d: projected %lld small-eig %lld ritz %lld correction %lld matvec %lld cycles\n",
           m, dits, dt[0], dt[1], dt[2], dt[3], dt[4]);
#endif
#undef DAV_T
  if (t == 0) {
    *pb.status = status;
    pb.lam[0] = theta;
  }
  for (int i = t; i < m; i += nt) pb.vec[i] = u[i];
  release();
}

}  // namespace

size_t eig_work_doubles(int64_t m) { return (size_t)eig_total_doubles(m); }

size_t davidson_work_doubles(int64_t m) {
  const int64_t ks = kDavMax;
  return (size_t)(3 * ks * m + 6 * m + 2 * ks * ks + eig_total_doubles(ks) + 2 + ks + 8 + 2 * m +
                  sizeof(DavCtl) / 8 + 8);
}

cudaError_t launch_davidson(const EigProblem* probs, double tol, int max_iter, double* work, int m,
                            cudaStream_t st) {
  static int grid = 0;
  const int smem = 200 * 1024;
  if (grid == 0) {
    cudaFuncSetAttribute(davidson_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, davidson_kernel, kEigThreads, smem);
    grid = sms * (per_sm > 0 ? per_sm : 1);
  }
  // the control block sits at the end of the problem's workspace
  DavCtl* ctl = reinterpret_cast<DavCtl*>(work + davidson_work_doubles(m) - sizeof(DavCtl) / 8 - 4);
  cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(DavCtl), st);
  if (e != cudaSuccess) return e;
  // a cooperative launch (every CTA resident: the grid barriers need it), written with the
  // launch-attribute form so that it can also be captured into a CUDA graph
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kEigThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, davidson_kernel, probs, tol, max_iter, ctl);
}

// per problem a team control block, then the queue counter
size_t eig_team_ctl_bytes(int nprob) {
  return sizeof(TeamCtl) * (size_t)(nprob > 0 ? nprob : 0) + 256;
}

// CTAs per problem (launches with fewer problems than SMs).  The estimated time of a problem of
// dimension d on T CTAs is
// d^3 (5 / T + 1): the FP64 reductions and eigenvectors (about 5 d^3 cycles on one CTA) are
// shared out, the QR (about d^3 with the FP32 location) is not.  Starting from one CTA each,
// the slowest problems get one more CTA together while the SMs last.
static std::vector<int> team_sizes(const int32_t* dims, int nprob, int sms) {
  std::vector<int> T(nprob, 1);
  auto est = [&](int p) { const double d = dims[p]; return d * d * d * (5.0 / T[p] + 1.0); };
  int budget = sms - nprob;
  while (budget > 0) {
    double mx = 0.0;
    for (int p = 0; p < nprob; ++p) mx = std::max(mx, est(p));
    std::vector<int> top;
    for (int p = 0; p < nprob; ++p)
      if (est(p) >= 0.98 * mx) top.push_back(p);
    bool can = (int)top.size() <= budget;
    for (int p : top) can = can && T[p] < kMaxTeam && dims[p] > kRows4Min;
    if (!can) break;
    for (int p : top) ++T[p];
    budget -= (int)top.size();
  }
  return T;
}

void launch_eig(const EigProblem* probs, int nprob, int threads, cudaStream_t st, const int32_t* dims,
                void* team_ctl) {
  if (nprob <= 0) return;
  (void)threads;
  const int smem = 200 * 1024;
  static int sms = 0;
  if (sms == 0) {
    cudaFuncSetAttribute(eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(eig_team_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(eig_team_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int dev = 0, n = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, eig_team_kernel<true>, kEigThreads, smem);
    sms = std::min(n * std::max(per_sm, 1), kTeamGridMax);
  }
  if (dims == nullptr || team_ctl == nullptr || nprob > kQueueMax) {
    eig_kernel<<<nprob, kEigThreads, smem, st>>>(probs);
    return;
  }
  auto est = [&](int p, int T) { const double d = dims[p]; return d * d * d * (5.0 / T + 1.0); };
  std::unique_ptr<TeamMap> mp(new TeamMap());   // (the launch parameter, staged on the host)
  TeamMap& map = *mp;
  int grid = 0;
  if (nprob < sms) {
    // every problem on its own CTAs
    const std::vector<int> T = team_sizes(dims, nprob, sms);
    for (int p = 0; p < nprob; ++p)
      for (int r = 0; r < T[p]; ++r, ++grid) {
        map.prob[grid] = (uint16_t)p;
        map.rank[grid] = (uint8_t)r;
        map.size[grid] = (uint8_t)T[p];
      }
    if (grid <= nprob) {
      eig_kernel<<<nprob, kEigThreads, smem, st>>>(probs);
      return;
    }
    map.nteam = grid;
  } else {
    // more problems than SMs: the ones slower than the balanced share of all the work get
    // teams (the smallest that bring them within it, at most kMaxTeam, half the SMs at most);
    // every CTA then works through the rest, largest first
    double total = 0.0;
    for (int p = 0; p < nprob; ++p) total += est(p, 1);
    const double share = total / sms;
    std::vector<int> order(nprob);
    for (int p = 0; p < nprob; ++p) order[p] = p;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return est(a, 1) > est(b, 1); });
    int c = 0;
    for (int p : order) {
      if (est(p, 1) <= share || dims[p] <= kRows4Min) {
        map.queue[map.nqueue++] = (uint16_t)p;
        continue;
      }
      int T = 2;
      while (T < kMaxTeam && est(p, T) > share) ++T;
      if (c + T > sms / 2) {
        map.queue[map.nqueue++] = (uint16_t)p;
        continue;
      }
      for (int r = 0; r < T; ++r, ++c) {
        map.prob[c] = (uint16_t)p;
        map.rank[c] = (uint8_t)r;
        map.size[c] = (uint8_t)T;
      }
    }
    map.nteam = c;
    grid = sms;
  }
  if (cudaMemsetAsync(team_ctl, 0, eig_team_ctl_bytes(nprob), st) != cudaSuccess) return;
  int* queue_head = reinterpret_cast<int*>(static_cast<char*>(team_ctl) + sizeof(TeamCtl) * (size_t)nprob);
  // a cooperative launch (every CTA resident: the team barriers need it), in the
  // launch-attribute form that stream capture accepts
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kEigThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (map.nqueue > 0)
    cudaLaunchKernelEx(&cfg, eig_team_kernel<true>, probs, reinterpret_cast<TeamCtl*>(team_ctl),
                       queue_head, map);
  else
    cudaLaunchKernelEx(&cfg, eig_team_kernel<false>, probs, reinterpret_cast<TeamCtl*>(team_ctl),
                       queue_head, map);
}

}  // namespace blm


// ---------------------------------------------------------------------------------------------
// Allocation-free block solve.
//
// Some callers cannot allocate device memory when they need a block solved: a VMC program that
// reserves the whole device for its walkers at start-up and then forbids further cudaMalloc,
// code that must not take the device-wide synchronisation that cudaMalloc/cudaFree can imply,
// or a host runtime that only hands this library pointers it already owns.  For them,
// blm_block_solve_noalloc runs the same dense solver as blm_block_solve on one block problem
// whose overlap and Hamiltonian the caller supplies, with its workspace in the file-scope array
// below (held by every GPU that loads the library until the process exits).
// ---------------------------------------------------------------------------------------------
namespace blm {
namespace {

constexpr int kNoAllocMaxDim = 257;     // block problems up to 1 + 256 parameters
constexpr int kNoAllocMaxKeep = 64;
constexpr size_t kNoAllocWork = (size_t)eig_total_doubles(kNoAllocMaxDim);
// workspace | eigenvectors (kNoAllocMaxKeep x kNoAllocMaxDim) | status word
constexpr size_t kNoAllocDoubles = kNoAllocWork + (size_t)kNoAllocMaxKeep * kNoAllocMaxDim + 8;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

__global__ void __launch_bounds__(kEigThreads)
noalloc_block_kernel(double* scratch, const double* S, const double* H, int dim, int keep,
                     double* lambda, double* B) {
  extern __shared__ double dsm[];
  __shared__ Shared sh;
  __shared__ double red[32];
  double* work = scratch;
  double* vec = scratch + kNoAllocWork;
  int32_t* status = reinterpret_cast<int32_t*>(vec + (size_t)kNoAllocMaxKeep * kNoAllocMaxDim);
  if (threadIdx.x == 0) *status = ST_OK;     // the array keeps the previous call's contents
  __syncthreads();
  EigProblem pb{dim, keep, 0, kEigLocate32, S, H, work, lambda, vec, status};
  dense_geig(pb, dsm, sh);
  __syncthreads();
  if (*status != ST_OK) return;
  // rows of B: beta parts of the eigenvectors, unit 2-norm, largest-magnitude entry positive
  const int m = dim - 1;
  for (int q = 0; q < keep; ++q) {
    const double* v = vec + (size_t)q * dim + 1;
    double part = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) part += v[i] * v[i];
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
      double n2 = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) n2 += red[w];
      int best = 0;
      for (int i = 1; i < m; ++i)
        if (fabs(v[i]) > fabs(v[best])) best = i;
      const bool ok = n2 > 0.0 && isfinite(n2);
      red[0] = ok ? (v[best] < 0.0 ? -1.0 : 1.0) / sqrt(n2) : 0.0;
      if (!ok) *status = ST_ZERO_DIR;
    }
    __syncthreads();
    const double sc = red[0];
    for (int i = threadIdx.x; i < m; i += blockDim.x) B[(size_t)q * m + i] = v[i] * sc;
    __syncthreads();
  }
}

}  // namespace

}  // namespace blm

#include <mutex>

namespace {
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[256] = {nullptr};
}  // namespace

extern "C" {

int32_t blm_noalloc_max_dim(void) { return blm::kNoAllocMaxDim; }

blm_status blm_block_solve_noalloc(const double* S, const double* H, int32_t dim,
                                   int32_t n_keep, double* lambda, double* B, void* stream) {
  if (!S || !H || !lambda || !B) return BLM_ERR_ARG;
  if (dim < 2 || dim > blm::kNoAllocMaxDim) {
    fprintf(stderr, "blm_block_solve_noalloc: dimension %d outside 2..%d (the static workspace "
                    "holds block problems up to %d)\n", dim, blm::kNoAllocMaxDim, blm::kNoAllocMaxDim);
    return BLM_ERR_ARG;
  }
  if (n_keep < 1 || n_keep > dim - 1 || n_keep > blm::kNoAllocMaxKeep) {
    fprintf(stderr, "blm_block_solve_noalloc: n_keep %d outside 1..%d\n", n_keep,
            dim - 1 < blm::kNoAllocMaxKeep ? dim - 1 : blm::kNoAllocMaxKeep);
    return BLM_ERR_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return BLM_ERR_CUDA;
  double* scratch = nullptr;
  {
    // once per device, with that device current: the array's device address
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, blm::g_noalloc_scratch) != cudaSuccess) {
        cudaGetLastError();
        return BLM_ERR_CUDA;
      }
      g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_noalloc_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int smem = 200 * 1024;
  if (cudaFuncSetAttribute(blm::noalloc_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           smem) != cudaSuccess)
    return BLM_ERR_CUDA;
  blm::noalloc_block_kernel<<<1, blm::kEigThreads, smem, st>>>(scratch, S, H, dim, n_keep,
                                                               lambda, B);
  if (cudaGetLastError() != cudaSuccess) return BLM_ERR_CUDA;
  int32_t status = 0;
  const int32_t* dstat = reinterpret_cast<const int32_t*>(
      scratch + blm::kNoAllocWork + (size_t)blm::kNoAllocMaxKeep * blm::kNoAllocMaxDim);
  if (cudaMemcpyAsync(&status, dstat, sizeof(status), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return BLM_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return BLM_ERR_CUDA;
  return status == blm::ST_OK ? BLM_OK : BLM_ERR_NUMERIC;
}

}  // extern "C"
