// FP64 generalized eigen-solver for the block problems (Eq. 5 / Eq. 10) and the combined problem
// (Eq. 7) of the blocked linear method: H v = lambda S v with H non-symmetric and S symmetric
// positive definite, keeping the eigenpairs with the lowest real parts (Sec. II.B).
//
// One CTA per problem (all blocks in one launch).  Steps, all FP64:
//   1. diagonal scaling  S~ = D S D, H~ = D H D with D = diag(S)^-1/2;
//   2. Cholesky  S~ = L L^T  and reduction to standard form  A = L^-1 H~ L^-T;
//   3. Householder reduction of A to upper Hessenberg form  A = Q Hs Q^T;
//   4. Francis double-shift QR on Hs for all eigenvalues (eigenvalues only, active window);
//   5. for each wanted eigenvalue, inverse iteration on the Hessenberg matrix (real or complex
//      LU with the one-row partial pivoting a Hessenberg matrix needs);
//   6. back-transformation  v = D L^-T Q y.
// Iterations are bounded: a QR that does not converge within 40 m sweeps reports ST_NOCONV.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>

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

// Banded upper-Hessenberg store used by the QR sweeps: row i keeps columns [max(0, i-3), m),
// room for the Hessenberg part plus the 3 x 3 bulge of a double-shift step.
struct Band {
  double* p;
  int m;
  __device__ __forceinline__ int64_t off(int i) const {
    if (i <= 4) return (int64_t)i * m;
    const int64_t r = i - 4;
    return 4LL * m + r * (m + 3) - (((int64_t)(i - 1) * i) / 2 - 6);
  }
  __device__ __forceinline__ double& at(int i, int j) const {
    const int c0 = i > 3 ? i - 3 : 0;
    return p[off(i) + (j - c0)];
  }
  __host__ __device__ static int64_t size(int m) {
    if (m <= 4) return (int64_t)m * m;
    const int64_t i = m, r = i - 4;
    return 4LL * m + r * (m + 3) - ((i - 1) * i / 2 - 6);
  }
};

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

// 3-vector (or 2-vector) Householder: returns beta, v = (1, v1, v2) with
// (I - beta v v^T) (x, y, z)^T = (alpha, 0, 0)^T.
__device__ void house3(double x, double y, double z, double& beta, double& v1, double& v2) {
  const double sigma = y * y + z * z;
  if (sigma == 0.0) {
    beta = 0.0;
    v1 = v2 = 0.0;
    return;
  }
  const double mu = sqrt(x * x + sigma);
  const double v0 = (x <= 0.0) ? (x - mu) : (-sigma / (x + mu));
  beta = 2.0 * v0 * v0 / (sigma + v0 * v0);
  v1 = y / v0;
  v2 = z / v0;
}

// Same banded store in another precision (FP32 for locating eigenvalues in shared memory).
template <typename R>
struct BandT {
  R* p;
  int m;
  __device__ __forceinline__ R& at(int i, int j) const {
    const int c0 = i > 3 ? i - 3 : 0;
    return p[Band{nullptr, m}.off(i) + (j - c0)];
  }
};

template <typename R>
__device__ __forceinline__ void house3t(R x, R y, R z, R& beta, R& v1, R& v2) {
  const R sigma = y * y + z * z;
  if (sigma == (R)0) {
    beta = v1 = v2 = (R)0;
    return;
  }
  const R mu = sqrt(x * x + sigma);
  const R v0 = (x <= (R)0) ? (x - mu) : (-sigma / (x + mu));
  beta = (R)2 * v0 * v0 / (sigma + v0 * v0);
  v1 = y / v0;
  v2 = z / v0;
}

// Francis double-shift QR for all eigenvalues, run by ONE warp on a banded store in shared
// memory: the scalar control (deflation search, shifts, reflectors) is computed redundantly by
// every lane, the row and column updates are split over the lanes.  Same algorithm as
// hqr_eigenvalues below; used in FP32 to locate eigenvalues that are then refined in FP64.
template <typename R>
__device__ bool hqr_warp(BandT<R> h, int m, double* wr, double* wi, R anorm) {
  const int lane = threadIdx.x & 31;
  const R eps = sizeof(R) == 4 ? (R)1.1920929e-7 : (R)2.220446049250313e-16;
  int hi = m - 1;
  int its = 0, total = 0;
  const int limit = 40 * m + 100;
  while (hi >= 0) {
    int l = hi;
    while (l > 0) {
      R s = fabs(h.at(l - 1, l - 1)) + fabs(h.at(l, l));
      if (s == (R)0) s = anorm;
      if (fabs(h.at(l, l - 1)) <= eps * s) break;
      --l;
    }
    __syncwarp();
    if (l > 0 && lane == 0) h.at(l, l - 1) = (R)0;
    __syncwarp();
    if (l == hi) {
      if (lane == 0) {
        wr[hi] = (double)h.at(hi, hi);
        wi[hi] = 0.0;
      }
      hi -= 1;
      its = 0;
      continue;
    }
    if (l == hi - 1) {
      if (lane == 0) {
        const double a = h.at(hi - 1, hi - 1), b = h.at(hi - 1, hi);
        const double c = h.at(hi, hi - 1), d = h.at(hi, hi);
        const double p = 0.5 * (a - d);
        const double disc = p * p + b * c;
        const double mid = 0.5 * (a + d);
        if (disc >= 0.0) {
          const double sq = sqrt(disc);
          wr[hi - 1] = mid - sq;
          wr[hi] = mid + sq;
          wi[hi - 1] = wi[hi] = 0.0;
        } else {
          const double sq = sqrt(-disc);
          wr[hi - 1] = wr[hi] = mid;
          wi[hi - 1] = sq;
          wi[hi] = -sq;
        }
      }
      hi -= 2;
      its = 0;
      continue;
    }
    if (total >= limit) return false;
    ++its;
    ++total;
    R sft, tt;
    if (its % 11 == 10) {
      const R e = fabs(h.at(hi, hi - 1)) + fabs(h.at(hi - 1, hi - 2));
      sft = (R)1.5 * e;
      tt = e * e;
    } else {
      sft = h.at(hi - 1, hi - 1) + h.at(hi, hi);
      tt = h.at(hi - 1, hi - 1) * h.at(hi, hi) - h.at(hi - 1, hi) * h.at(hi, hi - 1);
    }
    const R h00 = h.at(l, l), h10 = h.at(l + 1, l), h01 = h.at(l, l + 1);
    const R h11 = h.at(l + 1, l + 1), h21 = h.at(l + 2, l + 1);
    R x = h00 * h00 + h01 * h10 - sft * h00 + tt;
    R y = h10 * (h00 + h11 - sft);
    R z = h10 * h21;
    for (int k = l; k <= hi - 1; ++k) {
      const bool three = (k <= hi - 2);
      R beta, v1, v2;
      house3t<R>(x, y, three ? z : (R)0, beta, v1, v2);
      if (!three) v2 = (R)0;
      if (beta != (R)0) {
        const int c0 = (k > l) ? k - 1 : l;
        for (int j = c0 + lane; j <= hi; j += 32) {
          R p = h.at(k, j) + v1 * h.at(k + 1, j);
          if (three) p += v2 * h.at(k + 2, j);
          p *= beta;
          h.at(k, j) -= p;
          h.at(k + 1, j) -= p * v1;
          if (three) h.at(k + 2, j) -= p * v2;
        }
        __syncwarp();
        if (lane == 0 && k > l) {
          h.at(k + 1, k - 1) = (R)0;
          if (three) h.at(k + 2, k - 1) = (R)0;
        }
        const int rmax = three ? min(k + 3, hi) : hi;
        for (int i = l + lane; i <= rmax; i += 32) {
          R p = h.at(i, k) + v1 * h.at(i, k + 1);
          if (three) p += v2 * h.at(i, k + 2);
          p *= beta;
          h.at(i, k) -= p;
          h.at(i, k + 1) -= p * v1;
          if (three) h.at(i, k + 2) -= p * v2;
        }
        __syncwarp();
      }
      if (k < hi - 1) {
        x = h.at(k + 1, k);
        y = h.at(k + 2, k);
        z = (k < hi - 2) ? h.at(k + 3, k) : (R)0;
      }
      __syncwarp();
    }
  }
  return true;
}

struct Shared {
  double red[32];
  double scal[8];
  int iscal[8];
  int sel_idx[kMaxKeep];
  int sel_part[kMaxKeep];   // 0 real, 1 real part of complex, 2 imaginary part of complex
};

// ---------------------------------------------------------------------------------------------
// QR iteration for all eigenvalues of the Hessenberg matrix in `h` (banded store).
// Returns false if it did not converge.
// ---------------------------------------------------------------------------------------------
__device__ bool hqr_eigenvalues(Band h, int m, double* wr, double* wi, double anorm, Shared& sh) {
  const int t = threadIdx.x, nt = blockDim.x;
  const double eps = 2.220446049250313e-16;
  int hi = m - 1;
  int its = 0, total = 0;
  const int limit = 40 * m + 100;
  while (hi >= 0) {
    // --- deflation search (thread 0), broadcast l ---
    if (t == 0) {
      int l = hi;
      while (l > 0) {
        double s = fabs(h.at(l - 1, l - 1)) + fabs(h.at(l, l));
        if (s == 0.0) s = anorm;
        if (fabs(h.at(l, l - 1)) <= eps * s) {
          h.at(l, l - 1) = 0.0;
          break;
        }
        --l;
      }
      sh.iscal[0] = l;
    }
    __syncthreads();
    const int l = sh.iscal[0];
    __syncthreads();
    if (l == hi) {
      if (t == 0) {
        wr[hi] = h.at(hi, hi);
        wi[hi] = 0.0;
      }
      hi -= 1;
      its = 0;
      __syncthreads();
      continue;
    }
    if (l == hi - 1) {
      if (t == 0) {
        const double a = h.at(hi - 1, hi - 1), b = h.at(hi - 1, hi);
        const double c = h.at(hi, hi - 1), d = h.at(hi, hi);
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
      hi -= 2;
      its = 0;
      __syncthreads();
      continue;
    }
    if (total >= limit) return false;
    ++its;
    ++total;
    // --- shifts and first column (thread 0) ---
    if (t == 0) {
      double s, tt;
      if (its % 11 == 10) {
        const double e = fabs(h.at(hi, hi - 1)) + fabs(h.at(hi - 1, hi - 2));
        s = 1.5 * e;
        tt = e * e;
      } else {
        s = h.at(hi - 1, hi - 1) + h.at(hi, hi);
        tt = h.at(hi - 1, hi - 1) * h.at(hi, hi) - h.at(hi - 1, hi) * h.at(hi, hi - 1);
      }
      const double h00 = h.at(l, l), h10 = h.at(l + 1, l), h01 = h.at(l, l + 1);
      const double h11 = h.at(l + 1, l + 1), h21 = h.at(l + 2, l + 1);
      sh.scal[0] = h00 * h00 + h01 * h10 - s * h00 + tt;
      sh.scal[1] = h10 * (h00 + h11 - s);
      sh.scal[2] = h10 * h21;
    }
    __syncthreads();
    double x = sh.scal[0], y = sh.scal[1], z = sh.scal[2];
    __syncthreads();
    for (int k = l; k <= hi - 1; ++k) {
      const bool three = (k <= hi - 2);
      if (t == 0) {
        double beta, v1, v2;
        house3(x, y, three ? z : 0.0, beta, v1, v2);
        sh.scal[3] = beta;
        sh.scal[4] = v1;
        sh.scal[5] = three ? v2 : 0.0;
      }
      __syncthreads();
      const double beta = sh.scal[3], v1 = sh.scal[4], v2 = sh.scal[5];
      if (beta != 0.0) {
        const int c0 = (k > l) ? k - 1 : l;
        for (int j = c0 + t; j <= hi; j += nt) {
          if (three) {
            double p = h.at(k, j) + v1 * h.at(k + 1, j) + v2 * h.at(k + 2, j);
            p *= beta;
            h.at(k, j) -= p;
            h.at(k + 1, j) -= p * v1;
            h.at(k + 2, j) -= p * v2;
          } else {
            double p = h.at(k, j) + v1 * h.at(k + 1, j);
            p *= beta;
            h.at(k, j) -= p;
            h.at(k + 1, j) -= p * v1;
          }
        }
        __syncthreads();
        if (t == 0 && k > l) {
          h.at(k + 1, k - 1) = 0.0;
          if (three) h.at(k + 2, k - 1) = 0.0;
        }
        const int rmax = three ? min(k + 3, hi) : hi;
        for (int i = l + t; i <= rmax; i += nt) {
          if (three) {
            double p = h.at(i, k) + v1 * h.at(i, k + 1) + v2 * h.at(i, k + 2);
            p *= beta;
            h.at(i, k) -= p;
            h.at(i, k + 1) -= p * v1;
            h.at(i, k + 2) -= p * v2;
          } else {
            double p = h.at(i, k) + v1 * h.at(i, k + 1);
            p *= beta;
            h.at(i, k) -= p;
            h.at(i, k + 1) -= p * v1;
          }
        }
      }
      __syncthreads();
      if (k < hi - 1) {
        x = h.at(k + 1, k);
        y = h.at(k + 2, k);
        z = (k < hi - 2) ? h.at(k + 3, k) : 0.0;
      }
      __syncthreads();
    }
  }
  return true;
}

// ---------------------------------------------------------------------------------------------
// Inverse iteration on the Hessenberg matrix Hh (row-major m x m) for eigenvalue lam (complex
// allowed).  Writes the eigenvector (re, im) into yr, yi.  W: 2 m^2 doubles of workspace.
// ---------------------------------------------------------------------------------------------
__device__ void hess_inverse_iteration(const double* Hh, int m, double lre, double lim,
                                       double anorm, double* W, double* yr, double* yi,
                                       double* piv_l_re, double* piv_l_im, int* piv_swap,
                                       Shared& sh) {
  const int t = threadIdx.x, nt = blockDim.x;
  const bool cx = (lim != 0.0);
  double* Ur = W;
  double* Ui = W + (int64_t)m * m;
  // perturb the shift slightly so that the LU is not exactly singular
  const double pert = anorm * 1e-14;
  const double sre = lre + pert;
  const double sim = lim;
  for (int64_t idx = t; idx < (int64_t)m * m; idx += nt) {
    const int i = (int)(idx / m), j = (int)(idx % m);
    double v = (j >= i - 1) ? Hh[idx] : 0.0;
    if (i == j) v -= sre;
    Ur[idx] = v;
    if (cx) Ui[idx] = (i == j) ? -sim : 0.0;
  }
  __syncthreads();
  // LU with partial pivoting between rows k and k+1
  for (int k = 0; k < m - 1; ++k) {
    if (t == 0) {
      cplx a = cmk(Ur[(int64_t)k * m + k], cx ? Ui[(int64_t)k * m + k] : 0.0);
      cplx b = cmk(Ur[(int64_t)(k + 1) * m + k], cx ? Ui[(int64_t)(k + 1) * m + k] : 0.0);
      int sw = cabs2(b) > cabs2(a) ? 1 : 0;
      if (sw) {
        const cplx tmp = a;
        a = b;
        b = tmp;
      }
      if (cabs2(a) == 0.0) a = cmk(pert, 0.0);
      const cplx l = cdiv(b, a);
      piv_swap[k] = sw;
      piv_l_re[k] = l.re;
      piv_l_im[k] = l.im;
    }
    __syncthreads();
    const int sw = piv_swap[k];
    const cplx l = cmk(piv_l_re[k], piv_l_im[k]);
    for (int j = k + t; j < m; j += nt) {
      const int64_t ik = (int64_t)k * m + j, ik1 = (int64_t)(k + 1) * m + j;
      cplx a = cmk(Ur[ik], cx ? Ui[ik] : 0.0);
      cplx b = cmk(Ur[ik1], cx ? Ui[ik1] : 0.0);
      if (sw) {
        const cplx tmp = a;
        a = b;
        b = tmp;
      }
      b = b - l * a;
      Ur[ik] = a.re;
      Ur[ik1] = b.re;
      if (cx) {
        Ui[ik] = a.im;
        Ui[ik1] = b.im;
      }
    }
    __syncthreads();
  }
  // right-hand side: start from a fixed vector; iterate solves
  for (int i = t; i < m; i += nt) {
    yr[i] = 1.0 + 0.1 * (double)((i * 7919) % 97) / 97.0;
    yi[i] = 0.0;
  }
  __syncthreads();
  for (int iter = 0; iter < 3; ++iter) {
    // forward: apply the row swaps and multipliers
    if (t == 0) {
      for (int k = 0; k < m - 1; ++k) {
        cplx a = cmk(yr[k], yi[k]), b = cmk(yr[k + 1], yi[k + 1]);
        if (piv_swap[k]) {
          const cplx tmp = a;
          a = b;
          b = tmp;
        }
        b = b - cmk(piv_l_re[k], piv_l_im[k]) * a;
        yr[k] = a.re;
        yi[k] = a.im;
        yr[k + 1] = b.re;
        yi[k + 1] = b.im;
      }
    }
    __syncthreads();
    // back substitution with U (column oriented)
    for (int k = m - 1; k >= 0; --k) {
      if (t == 0) {
        cplx d = cmk(Ur[(int64_t)k * m + k], cx ? Ui[(int64_t)k * m + k] : 0.0);
        if (cabs2(d) == 0.0) d = cmk(pert, 0.0);
        const cplx xk = cdiv(cmk(yr[k], yi[k]), d);
        yr[k] = xk.re;
        yi[k] = xk.im;
      }
      __syncthreads();
      const cplx xk = cmk(yr[k], yi[k]);
      for (int i = t; i < k; i += nt) {
        const cplx u = cmk(Ur[(int64_t)i * m + k], cx ? Ui[(int64_t)i * m + k] : 0.0);
        const cplx v = cmk(yr[i], yi[i]) - u * xk;
        yr[i] = v.re;
        yi[i] = v.im;
      }
      __syncthreads();
    }
    // normalise (max-abs)
    double mx = 0.0;
    for (int i = t; i < m; i += nt) mx = fmax(mx, fabs(yr[i]) + fabs(yi[i]));
    mx = block_max(mx, sh.red);
    const double inv = mx > 0.0 ? 1.0 / mx : 1.0;
    for (int i = t; i < m; i += nt) {
      yr[i] *= inv;
      yi[i] *= inv;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------
// Per-warp eigenvector refinement (no CTA barriers).  One warp runs Rayleigh-quotient iteration
// on the FP64 Hessenberg matrix Hh for the eigenvalue nearest (sre, sim): each round factors
// (Hh - sigma I) = P L U with the one-row pivoting a Hessenberg matrix needs, solves twice from
// the current vector, and updates sigma to the Rayleigh quotient x^H Hh x / x^H x.  Rows being
// eliminated live in shared memory (cur, nxt); U is stored packed (row k holds columns k..m-1).
// CX selects complex arithmetic (complex shift) at compile time.
// ---------------------------------------------------------------------------------------------
constexpr int kRqiWarps = 8;
constexpr int kMaxCand = 64;

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
    const cplx lm = CX ? cdiv(b, a) : cmk(b.re / a.re, 0.0);
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
      const cplx x = CX ? cdiv(num, d) : cmk(num.re / d.re, 0.0);
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

// out = Hh x for a real vector x (one warp; out written by lane 0 row by row).
__device__ void warp_hess_matvec(const double* Hh, int m, const double* x, double* out) {
  const int lane = threadIdx.x & 31;
  for (int i = 0; i < m; ++i) {
    const double* hrow = Hh + (int64_t)i * m;
    double h = 0.0;
    for (int j = (i > 0 ? i - 1 : 0) + lane; j < m; j += 32) h = fma(hrow[j], x[j], h);
    h = warp_sum(h);
    if (lane == 0) out[i] = h;
  }
  __syncwarp();
}

__device__ double warp_dot(const double* a, const double* b, int m) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int i = lane; i < m; i += 32) s = fma(a[i], b[i], s);
  return warp_sum(s);
}

// Rayleigh-quotient iteration for the eigenvalue nearest (sre, sim): the first round solves
// four times at the given shift (two when a start vector is supplied in yv), later rounds two
// times at the updated Rayleigh quotient; stops when ||Hh x - lambda x|| <= 1e-11 ||Hh|| ||x||.
template <bool CX>
__device__ bool warp_rqi(const double* Hh, int m, double anorm, double& sre, double& sim,
                         int max_rounds, double* cur, double* nxt, double* yv, double* U,
                         double* pl, int* ps, bool have_start = false) {
  const int lane = threadIdx.x & 31;
  const double pert = anorm * 1e-14;   // keeps the factorisation nonsingular at an eigenvalue
  if (!have_start) {
    for (int i = lane; i < m; i += 32) {
      yv[i] = 1.0 + 0.1 * (double)((i * 7919) % 97) / 97.0;
      yv[m + i] = 0.0;
    }
  }
  __syncwarp();
  bool converged = false;
  for (int round = 0; round < max_rounds && !converged; ++round) {
    warp_hess_lu<CX>(Hh, m, sre + pert, CX ? sim : 0.0, pert, cur, nxt, U, pl, ps);
    const int nsolve = (round == 0 && !have_start) ? 4 : 2;
    for (int it = 0; it < nsolve; ++it) warp_hess_solve<CX>(m, pert, U, pl, ps, yv);
    // Hx into cur (free now), Rayleigh quotient, residual
    for (int i = 0; i < m; ++i) {
      const double* hrow = Hh + (int64_t)i * m;
      double hr = 0.0, hi = 0.0;
      for (int j = (i > 0 ? i - 1 : 0) + lane; j < m; j += 32) {
        hr = fma(hrow[j], yv[j], hr);
        if (CX) hi = fma(hrow[j], yv[m + j], hi);
      }
      hr = warp_sum(hr);
      if (CX) hi = warp_sum(hi);
      if (lane == 0) {
        cur[i] = hr;
        cur[m + i] = hi;
      }
    }
    __syncwarp();
    double pr = 0.0, pi = 0.0, pn = 0.0;
    for (int i = lane; i < m; i += 32) {
      const double xr = yv[i], xi = CX ? yv[m + i] : 0.0;
      pr += xr * cur[i] + xi * cur[m + i];
      pi += xr * cur[m + i] - xi * cur[i];
      pn += xr * xr + xi * xi;
    }
    pr = warp_sum(pr);
    if (CX) pi = warp_sum(pi);
    pn = warp_sum(pn);
    sre = pr / pn;
    if (CX) sim = pi / pn;
    double rr = 0.0;
    for (int i = lane; i < m; i += 32) {
      const double xr = yv[i], xi = CX ? yv[m + i] : 0.0;
      const double er = cur[i] - (sre * xr - (CX ? sim * xi : 0.0));
      const double ei = CX ? cur[m + i] - (sre * xi + sim * xr) : 0.0;
      rr += er * er + ei * ei;
    }
    rr = warp_sum(rr);
    converged = sqrt(rr) <= 1e-11 * anorm * sqrt(pn);
    __syncwarp();
  }
  return converged;
}

// Two close eigenvalues near the real shift sigma (a near-degenerate real pair, or a complex
// pair): subspace iteration with two vectors at sigma, a 2 x 2 Rayleigh-Ritz step on the
// converged invariant plane, then Rayleigh-quotient polishing of each Ritz pair.  Writes up to
// two results (re, im, vector re|im of length 2m); a complex pair is one result (+ member).
// Returns the number of converged results.
__device__ int warp_pair(const double* Hh, int m, double anorm, double sigma, double* cur,
                         double* nxt, double* yv, double* U, double* pl, int* ps,
                         double* ore, double* oim, double* v0, double* v1) {
  const int lane = threadIdx.x & 31;
  const double pert = anorm * 1e-14;
  double* y1 = yv;
  double* y2 = yv + m;
  for (int i = lane; i < m; i += 32) {
    y1[i] = 1.0 + 0.1 * (double)((i * 7919) % 97) / 97.0;
    y2[i] = 1.0 - 0.3 * (double)((i * 104729) % 89) / 89.0;
  }
  __syncwarp();
  warp_hess_lu<false>(Hh, m, sigma + pert, 0.0, pert, cur, nxt, U, pl, ps);
  for (int it = 0; it < 6; ++it) {
    warp_hess_solve<false>(m, pert, U, pl, ps, y1);
    warp_hess_solve<false>(m, pert, U, pl, ps, y2);
    for (int pass = 0; pass < 2; ++pass) {
      const double n1 = sqrt(warp_dot(y1, y1, m));
      for (int i = lane; i < m; i += 32) y1[i] /= n1;
      __syncwarp();
      const double c = warp_dot(y1, y2, m);
      for (int i = lane; i < m; i += 32) y2[i] -= c * y1[i];
      __syncwarp();
      const double n2 = sqrt(warp_dot(y2, y2, m));
      for (int i = lane; i < m; i += 32) y2[i] /= n2;
      __syncwarp();
    }
  }
  // T = Y^T Hh Y
  warp_hess_matvec(Hh, m, y1, cur);
  warp_hess_matvec(Hh, m, y2, cur + m);
  const double t11 = warp_dot(y1, cur, m), t21 = warp_dot(y2, cur, m);
  const double t12 = warp_dot(y1, cur + m, m), t22 = warp_dot(y2, cur + m, m);
  const double tr = 0.5 * (t11 + t22), det = t11 * t22 - t12 * t21;
  const double disc = tr * tr - det;
  // Ritz vectors into v0 / v1 (re | im), from z = (t12, mu - t11) or (mu - t22, t21)
  int nres = 0;
  if (disc >= 0.0) {
    const double sq = sqrt(disc);
    const double mus[2] = {tr - sq, tr + sq};
    for (int r = 0; r < 2; ++r) {
      const double mu = mus[r];
      double z1 = t12, z2 = mu - t11;
      if (fabs(mu - t22) + fabs(t21) > fabs(z1) + fabs(z2)) {
        z1 = mu - t22;
        z2 = t21;
      }
      double* out = r == 0 ? v0 : v1;
      for (int i = lane; i < m; i += 32) {
        out[i] = z1 * y1[i] + z2 * y2[i];
        out[m + i] = 0.0;
      }
      __syncwarp();
      ore[r] = mu;
      oim[r] = 0.0;
    }
    nres = 2;
  } else {
    const double im = sqrt(-disc);
    // mu = tr + i im;  z = (t12, mu - t11) complex
    const double z1r = t12, z1i = 0.0, z2r = tr - t11, z2i = im;
    for (int i = lane; i < m; i += 32) {
      v0[i] = z1r * y1[i] + z2r * y2[i];
      v0[m + i] = z1i * y1[i] + z2i * y2[i];
    }
    __syncwarp();
    ore[0] = tr;
    oim[0] = im;
    nres = 1;
  }
  // polish each Ritz pair
  int nconv = 0;
  for (int r = 0; r < nres; ++r) {
    double* out = r == 0 ? v0 : v1;
    for (int i = lane; i < 2 * m; i += 32) yv[i] = out[i];
    __syncwarp();
    double lre = ore[r], lim = oim[r];
    const bool conv = (lim != 0.0)
                          ? warp_rqi<true>(Hh, m, anorm, lre, lim, 3, cur, nxt, yv, U, pl, ps, true)
                          : warp_rqi<false>(Hh, m, anorm, lre, lim, 3, cur, nxt, yv, U, pl, ps, true);
    for (int i = lane; i < 2 * m; i += 32) out[i] = (lim != 0.0 || i < m) ? yv[i] : 0.0;
    __syncwarp();
    ore[r] = lre;
    oim[r] = conv ? (fabs(lim) <= 1e-10 * fmax(1.0, fabs(lre)) ? 0.0 : fabs(lim)) : -1.0;
    nconv += conv ? 1 : 0;
  }
  return nconv;
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

// v <- D L^-T Q v  for a real vector v (Q from the stored Householder vectors in A).
__device__ void back_transform(const double* A, const double* hbeta, const double* L,
                               const double* dsc, int m, double* v, Shared& sh) {
  const int t = threadIdx.x, nt = blockDim.x;
  // Q = P_0 P_1 ... P_{m-3}; apply P_{m-3} first.  P_k acts on indices k+1..m-1 with
  // u = (1, A[k+2][k], ..., A[m-1][k]).
  for (int k = m - 3; k >= 0; --k) {
    const double beta = hbeta[k];
    if (beta == 0.0) continue;
    double part = 0.0;
    for (int i = k + 1 + t; i < m; i += nt) {
      const double u = (i == k + 1) ? 1.0 : A[(int64_t)i * m + k];
      part += u * v[i];
    }
    const double dot = block_sum(part, sh.red);
    for (int i = k + 1 + t; i < m; i += nt) {
      const double u = (i == k + 1) ? 1.0 : A[(int64_t)i * m + k];
      v[i] -= beta * dot * u;
    }
    __syncthreads();
  }
  // z = L^-T v  (L lower, row-major): for i = m-1..0: z_i = v_i / L_ii; v_j -= L_ij z_i (j < i)
  for (int i = m - 1; i >= 0; --i) {
    if (t == 0) v[i] = v[i] / L[(int64_t)i * m + i];
    __syncthreads();
    const double zi = v[i];
    for (int j = t; j < i; j += nt) v[j] -= L[(int64_t)i * m + j] * zi;
    __syncthreads();
  }
  for (int i = t; i < m; i += nt) v[i] *= dsc[i];
  __syncthreads();
}

// Dense solver for one problem, run by the whole CTA (dsm: up to 200 KB of shared memory).
__device__ void dense_geig(const EigProblem pb, double* dsm, Shared& sh) {
  const int m = pb.m;
  const int t = threadIdx.x, nt = blockDim.x;
  const int64_t mm = (int64_t)m * m;
  double* L = pb.work;
  double* A = L + mm;
  double* Hh = A + mm;
  double* W = Hh + mm;            // 2 m^2 (band store for QR, then LU workspace)
  double* dsc = W + 2 * mm;
  double* hbeta = dsc + m;
  double* wr = hbeta + m;
  double* wi = wr + m;
  double* yr = wi + m;
  double* yi = yr + m;
  double* col = yi + m;           // m
  double* plr = col + m;
  double* pli = plr + m;
  int* pswap = reinterpret_cast<int*>(pli + m);
  double* vtmp = pli + 2 * m;     // m

  if (t == 0) sh.iscal[1] = ST_OK;
  __syncthreads();
  // ---- 1. scaling ----
  for (int i = t; i < m; i += nt) {
    const double s = pb.S[(int64_t)i * m + i];
    if (!(s > 0.0) || !isfinite(s)) sh.iscal[1] = ST_NOT_PD;
    dsc[i] = (s > 0.0) ? 1.0 / sqrt(s) : 0.0;
  }
  __syncthreads();
  if (sh.iscal[1] != ST_OK) {
    if (t == 0) *pb.status = sh.iscal[1];
    return;
  }
  for (int64_t idx = t; idx < mm; idx += nt) {
    const int i = (int)(idx / m), j = (int)(idx % m);
    const double sv = pb.S[idx] * dsc[i] * dsc[j];
    const double hv = pb.H[idx] * dsc[i] * dsc[j];
    if (!isfinite(sv) || !isfinite(hv)) sh.iscal[1] = ST_NONFINITE;
    L[idx] = sv;
    A[idx] = hv;
  }
  __syncthreads();
  if (sh.iscal[1] != ST_OK) {
    if (t == 0) *pb.status = sh.iscal[1];
    return;
  }
  // ---- 2a. Cholesky (right-looking, lower) ----
  for (int k = 0; k < m; ++k) {
    if (t == 0) {
      const double p = L[(int64_t)k * m + k];
      if (!(p > 1e-15)) {
        sh.iscal[1] = ST_NOT_PD;
      } else {
        L[(int64_t)k * m + k] = sqrt(p);
        sh.scal[0] = 1.0 / sqrt(p);
      }
    }
    __syncthreads();
    if (sh.iscal[1] != ST_OK) break;
    const double inv = sh.scal[0];
    for (int i = k + 1 + t; i < m; i += nt) {
      const double v = L[(int64_t)i * m + k] * inv;
      L[(int64_t)i * m + k] = v;
      col[i] = v;
    }
    __syncthreads();
    const int r = m - k - 1;
    for (int64_t idx = t; idx < (int64_t)r * r; idx += nt) {
      const int ii = (int)(idx / r), jj = (int)(idx % r);
      if (jj <= ii) {
        const int i = k + 1 + ii, j = k + 1 + jj;
        L[(int64_t)i * m + j] -= col[i] * col[j];
      }
    }
    __syncthreads();
  }
  if (sh.iscal[1] != ST_OK) {
    if (t == 0) *pb.status = sh.iscal[1];
    return;
  }
  // ---- 2b. A <- L^-1 A (row forward substitution) ----
  for (int k = 0; k < m; ++k) {
    const double inv = 1.0 / L[(int64_t)k * m + k];
    for (int j = t; j < m; j += nt) {
      const double v = A[(int64_t)k * m + j] * inv;
      A[(int64_t)k * m + j] = v;
      col[j] = v;
    }
    __syncthreads();
    const int r = m - k - 1;
    for (int64_t idx = t; idx < (int64_t)r * m; idx += nt) {
      const int i = k + 1 + (int)(idx / m), j = (int)(idx % m);
      A[(int64_t)i * m + j] -= L[(int64_t)i * m + k] * col[j];
    }
    __syncthreads();
  }
  // ---- 2c. A <- A L^-T (column forward substitution) ----
  for (int k = 0; k < m; ++k) {
    const double inv = 1.0 / L[(int64_t)k * m + k];
    for (int i = t; i < m; i += nt) {
      const double v = A[(int64_t)i * m + k] * inv;
      A[(int64_t)i * m + k] = v;
      col[i] = v;
    }
    __syncthreads();
    const int r = m - k - 1;
    for (int64_t idx = t; idx < (int64_t)m * r; idx += nt) {
      const int i = (int)(idx / r), j = k + 1 + (int)(idx % r);
      A[(int64_t)i * m + j] -= L[(int64_t)j * m + k] * col[i];
    }
    __syncthreads();
  }
  // ---- 3. Householder reduction to Hessenberg form ----
  for (int k = 0; k < m - 2; ++k) {
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
    if (t == 0) hbeta[k] = beta;
    // u = (1, x[1:]/v0) into col[k+1..m-1]
    for (int i = k + 1 + t; i < m; i += nt) col[i] = (i == k + 1) ? 1.0 : A[(int64_t)i * m + k] / v0;
    __syncthreads();
    if (beta != 0.0) {
      // left: rows k+1.., columns k.. (column-owned)
      for (int j = k + t; j < m; j += nt) {
        double wj = 0.0;
        for (int i = k + 1; i < m; ++i) wj += col[i] * A[(int64_t)i * m + j];
        wj *= beta;
        for (int i = k + 1; i < m; ++i) A[(int64_t)i * m + j] -= wj * col[i];
      }
      __syncthreads();
      // right: all rows, columns k+1.. (warp per row)
      const int lane = t & 31, wid = t >> 5, nw = nt >> 5;
      for (int i = wid; i < m; i += nw) {
        double zi = 0.0;
        for (int j = k + 1 + lane; j < m; j += 32) zi += A[(int64_t)i * m + j] * col[j];
        for (int o = 16; o > 0; o >>= 1) zi += __shfl_xor_sync(0xffffffffu, zi, o);
        zi *= beta;
        for (int j = k + 1 + lane; j < m; j += 32) A[(int64_t)i * m + j] -= zi * col[j];
      }
      __syncthreads();
    }
    // store the reflector below the subdiagonal
    for (int i = k + 2 + t; i < m; i += nt) A[(int64_t)i * m + k] = col[i];
    __syncthreads();
  }
  // ---- Hessenberg copies: Hh (full) and the band store in shared or global memory ----
  double amx = 0.0;
  for (int64_t idx = t; idx < mm; idx += nt) {
    const int i = (int)(idx / m), j = (int)(idx % m);
    const double v = (j >= i - 1) ? A[idx] : 0.0;
    Hh[idx] = v;
    amx = fmax(amx, fabs(v));
  }
  const double anorm = fmax(block_max(amx, sh.red), 1e-300);
  const int64_t bsize = Band::size(m);
  const int want = pb.mode == 1 ? 1 : pb.k;
  // ---- 4. eigenvalues ----
  // Large problems whose FP64 band does not fit in shared memory: locate all eigenvalues with an
  // FP32 QR (one warp, band in shared memory), then refine the lowest candidates in FP64 by
  // Hessenberg inverse iteration and Rayleigh quotients; the rest are excluded (+inf).  Two
  // candidates that refine to the same eigenvalue mean the location was too coarse: the FP64 QR
  // below then runs instead.
  bool located = false;
  // extra workspace beyond 5 m^2 + 16 m (see eig_work_doubles)
  double* xbase = pb.work + 5 * mm + 16 * (int64_t)m;
  double* Uw = xbase;                                          // kRqiWarps x m(m+1)
  double* plw = Uw + (int64_t)kRqiWarps * m * (m + 1);         // kRqiWarps x 2m
  int* psw = reinterpret_cast<int*>(plw + (int64_t)kRqiWarps * 2 * m);   // kRqiWarps x m ints
  double* cvec = plw + (int64_t)kRqiWarps * 3 * m;             // kMaxCand x 2m
  double* cre = cvec + (int64_t)kMaxCand * 2 * m;              // kMaxCand
  double* cim = cre + kMaxCand;                                // kMaxCand
  if (bsize * 8 > (int64_t)200 * 1024 && bsize * 4 <= (int64_t)200 * 1024 && m <= 533 &&
      want + 8 <= kMaxCand && m > 2 * (want + 8)) {
    BandT<float> b32{reinterpret_cast<float*>(dsm), m};
    for (int i = t; i < m; i += nt) {
      const int c0 = i > 3 ? i - 3 : 0;
      for (int j = c0; j < m; ++j) b32.at(i, j) = (j >= i - 1) ? (float)Hh[(int64_t)i * m + j] : 0.0f;
    }
    __syncthreads();
    if (t < 32) {
      const bool ok32 = hqr_warp<float>(b32, m, wr, wi, (float)anorm);
      if (t == 0) sh.iscal[3] = ok32 ? 1 : 0;
#ifdef BLM_EIG_DEBUG
      if (t == 0 && !ok32) printf("eig: FP32 QR did not converge (m=%d)\n", m);
#endif
    }
    __syncthreads();
    if (sh.iscal[3]) {
      // Candidates, lowest FP32 real parts first, until want + 8 eigenvalues are covered.  A real
      // FP32 eigenvalue gives one real candidate.  A complex FP32 pair a +- ib gives a complex
      // candidate; when b is small the pair may be two close real eigenvalues that FP32 rounding
      // turned complex (square-root sensitivity), so real candidates at a - |b| and a + |b| are
      // added.  Each candidate is refined by Rayleigh-quotient iteration and kept only if its
      // FP64 residual is small; results are merged, and the refined eigenvalues below the cut are
      // counted against the FP32 ones there before they are trusted.
      if (t == 0) {
        for (int i = 0; i < m; ++i) vtmp[i] = 0.0;
        int slots = 0, nc = 0;
        while (slots < want + 8 && nc + 3 <= kMaxCand) {
          int best = -1;
          double bv = 0.0;
          for (int i = 0; i < m; ++i)
            if (vtmp[i] == 0.0 && (best < 0 || wr[i] < bv)) {
              best = i;
              bv = wr[i];
            }
          if (best < 0) break;
          vtmp[best] = 1.0;
          if (wi[best] != 0.0) {
            int partner = -1;
            if (best + 1 < m && wi[best + 1] == -wi[best]) partner = best + 1;
            if (best > 0 && wi[best - 1] == -wi[best]) partner = best - 1;
            if (partner >= 0) vtmp[partner] = 1.0;
            const double a = wr[best], b = fabs(wi[best]);
            cre[nc] = a;
            cim[nc] = b;
            ++nc;
            if (b <= 1e-2 * fmax(1.0, fabs(a))) {
              cre[nc] = a - b;
              cim[nc] = 0.0;
              ++nc;
              cre[nc] = a + b;
              cim[nc] = 0.0;
              ++nc;
            }
            slots += 2;
          } else {
            cre[nc] = wr[best];
            cim[nc] = 0.0;
            ++nc;
            slots += 1;
          }
        }
        sh.iscal[4] = nc;
      }
      __syncthreads();
      const int nc = sh.iscal[4];
      // Rayleigh-quotient iteration, one warp per candidate; cim < 0 marks "not converged"
      const int warp = t >> 5, lane = t & 31;
      if (warp < kRqiWarps) {
        double* cur = dsm + (int64_t)warp * 6 * m;
        double* nxt = cur + 2 * m;
        double* yv = nxt + 2 * m;
        double* U = Uw + (int64_t)warp * m * (m + 1);
        double* pl = plw + (int64_t)warp * 2 * m;
        int* ps = psw + (int64_t)warp * m;
        for (int c = warp; c < nc; c += kRqiWarps) {
          double lre = cre[c], lim = cim[c];
          const bool conv = (lim != 0.0)
                                ? warp_rqi<true>(Hh, m, anorm, lre, lim, 8, cur, nxt, yv, U, pl, ps)
                                : warp_rqi<false>(Hh, m, anorm, lre, lim, 8, cur, nxt, yv, U, pl, ps);
          for (int i = lane; i < m; i += 32) {
            cvec[(int64_t)c * 2 * m + i] = yv[i];
            cvec[(int64_t)c * 2 * m + m + i] = (lim != 0.0) ? yv[m + i] : 0.0;
          }
          if (lane == 0) {
            const bool real = fabs(lim) <= 1e-10 * fmax(1.0, fabs(lre));
            cre[c] = lre;
            cim[c] = conv ? (real ? 0.0 : fabs(lim)) : -1.0;
          }
          __syncwarp();
        }
      }
      __syncthreads();
      // Second pass: a candidate that did not converge, or two that converged to one value,
      // mark a close pair (or a complex pair) that single-vector iteration cannot separate;
      // those get the two-vector cluster refinement.
      if (t == 0) {
        int njobs = 0, next = nc;
        for (int c = 0; c < kMaxCand; ++c) vtmp[c] = 0.0;
        for (int a = 0; a < nc && njobs < kMaxKeep; ++a) {
          if (vtmp[a] != 0.0) continue;
          int partner = -1;
          if (cim[a] < 0.0) {
            if (next < kMaxCand) {
              partner = next++;
              cim[partner] = -1.0;
            }
          } else {
            for (int b = a + 1; b < nc; ++b)
              if (vtmp[b] == 0.0 && cim[b] >= 0.0 &&
                  fabs(cre[a] - cre[b]) + fabs(cim[a] - cim[b]) <= 1e-9 * fmax(1.0, fabs(cre[a]))) {
                partner = b;
                break;
              }
          }
          if (partner < 0) continue;
          vtmp[a] = vtmp[partner] = 1.0;
          sh.sel_idx[njobs] = a;
          sh.sel_part[njobs] = partner;
          ++njobs;
        }
        sh.iscal[5] = njobs;
        sh.iscal[4] = next;
      }
      __syncthreads();
      {
        const int njobs = sh.iscal[5];
        if (warp < kRqiWarps) {
          double* cur = dsm + (int64_t)warp * 6 * m;
          double* nxt = cur + 2 * m;
          double* yv = nxt + 2 * m;
          double* U = Uw + (int64_t)warp * m * (m + 1);
          double* pl = plw + (int64_t)warp * 2 * m;
          int* ps = psw + (int64_t)warp * m;
          for (int j = warp; j < njobs; j += kRqiWarps) {
            const int a = sh.sel_idx[j], b = sh.sel_part[j];
            double ore[2] = {0.0, 0.0}, oim[2] = {-1.0, -1.0};
            warp_pair(Hh, m, anorm, cre[a], cur, nxt, yv, U, pl, ps, ore, oim,
                      cvec + (int64_t)a * 2 * m, cvec + (int64_t)b * 2 * m);
            if (lane == 0) {
              cre[a] = ore[0];
              cim[a] = oim[0];
              cre[b] = ore[1];
              cim[b] = oim[1];
            }
            __syncwarp();
          }
        }
      }
      __syncthreads();
      const int nc2 = sh.iscal[4];
      if (t == 0) {
        const int nc = nc2;
        // merge: keep the first converged candidate of each distinct eigenvalue (flag 1.0)
        for (int c = 0; c < nc; ++c) vtmp[c] = (cim[c] >= 0.0) ? 1.0 : 0.0;
        for (int a = 0; a < nc; ++a) {
          if (vtmp[a] == 0.0) continue;
          for (int b = a + 1; b < nc; ++b)
            if (vtmp[b] != 0.0 &&
                fabs(cre[a] - cre[b]) + fabs(cim[a] - cim[b]) <= 1e-9 * fmax(1.0, fabs(cre[a])))
              vtmp[b] = 0.0;
        }
        // choose the want lowest distinct eigenvalues
        int nsel = 0;
        double cut_lo = -INFINITY;
        while (nsel < want) {
          int best = -1;
          for (int c = 0; c < nc; ++c)
            if (vtmp[c] == 1.0 && (best < 0 || cre[c] < cre[best])) best = c;
          if (best < 0) break;
          vtmp[best] = 2.0;
          cut_lo = cre[best];
          sh.sel_idx[nsel] = best;
          sh.sel_part[nsel] = cim[best] != 0.0 ? 1 : 0;
          ++nsel;
          if (cim[best] != 0.0 && nsel < want) {
            sh.sel_idx[nsel] = best;
            sh.sel_part[nsel] = 2;
            ++nsel;
          }
        }
        // completeness: count eigenvalues strictly below the midpoint between the last chosen
        // and the next refined one, among the refined (pairs count 2) and among the FP32 set
        double cut_hi = INFINITY;
        for (int c = 0; c < nc; ++c)
          if (vtmp[c] == 1.0 && cre[c] > cut_lo && cre[c] < cut_hi) cut_hi = cre[c];
        int ok = (nsel == want) && (cut_hi < INFINITY) && (cut_hi - cut_lo > 1e-9 * fmax(1.0, fabs(cut_lo)));
        if (ok) {
          const double cut = 0.5 * (cut_lo + cut_hi);
          int n_ref = 0, n_fp32 = 0;
          for (int c = 0; c < nc; ++c)
            if (vtmp[c] != 0.0 && cre[c] < cut) n_ref += cim[c] != 0.0 ? 2 : 1;
          for (int i = 0; i < m; ++i)
            if (wr[i] < cut) ++n_fp32;
          ok = (n_ref == n_fp32);
#ifdef BLM_EIG_DEBUG
          if (!ok) printf("eig: block %d count mismatch below %.9f: refined %d, fp32 %d\n", (int)blockIdx.x, cut, n_ref, n_fp32);
#endif
        }
        if (pb.mode == 1 && ok && sh.sel_part[0] != 0) sh.iscal[1] = ST_COMPLEX;
        sh.iscal[3] = ok ? 1 : 0;
        sh.iscal[2] = nsel;
#ifdef BLM_EIG_DEBUG
        if (!ok) {
          printf("eig: refined candidates incomplete (m=%d, nc=%d, nsel=%d)\n", m, nc, nsel);
          for (int c = 0; c < nc; ++c) printf("  cand %d: %.12f %+.3e\n", c, cre[c], cim[c]);
        }
#endif
      }
      // Householder vectors as rows for coalesced per-warp back-transformation (W is free here)
      for (int64_t idx = t; idx < mm; idx += nt) {
        const int k = (int)(idx / m), i = (int)(idx % m);
        W[idx] = (i >= k + 2 && k < m - 2) ? A[(int64_t)i * m + k] : 0.0;
      }
      __syncthreads();
      located = sh.iscal[3] != 0;
      if (located) {
        if (sh.iscal[1] != ST_OK) {
          if (t == 0) *pb.status = sh.iscal[1];
          return;
        }
        const int nsel = sh.iscal[2];
        const int nw = nt >> 5;
        for (int q = warp; q < nsel; q += nw) {
          const int c = sh.sel_idx[q], part = sh.sel_part[q];
          double* vr2 = dsm + (int64_t)warp * 2 * m;
          double* vi2 = vr2 + m;
          for (int i = lane; i < m; i += 32) {
            vr2[i] = cvec[(int64_t)c * 2 * m + i];
            vi2[i] = cvec[(int64_t)c * 2 * m + m + i];
          }
          __syncwarp();
          warp_back_transform(W, hbeta, L, dsc, m, vr2);
          if (part) {
            warp_back_transform(W, hbeta, L, dsc, m, vi2);
            // phase: largest-magnitude component real and positive
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
              vr2[i] = a2 * cc + b2 * ss;
              vi2[i] = b2 * cc - a2 * ss;
            }
            __syncwarp();
          }
          double* out = pb.vec + (int64_t)q * m;
          const double* src = (part == 2) ? vi2 : vr2;
          for (int i = lane; i < m; i += 32) out[i] = src[i];
          if (lane == 0) pb.lam[q] = cre[c];
          __syncwarp();
        }
        __syncthreads();
        if (t == 0) *pb.status = ST_OK;
        return;
      }
    }
  }
  if (!located) {
    const bool in_smem = (bsize * 8 <= (int64_t)200 * 1024);
    Band band{in_smem ? dsm : W, m};
    for (int i = t; i < m; i += nt) {
      const int c0 = i > 3 ? i - 3 : 0;
      for (int j = c0; j < m; ++j) band.at(i, j) = (j >= i - 1) ? Hh[(int64_t)i * m + j] : 0.0;
    }
    __syncthreads();
    const bool ok = hqr_eigenvalues(band, m, wr, wi, anorm, sh);
    __syncthreads();
    if (!ok) {
      if (t == 0) *pb.status = ST_NOCONV;
      return;
    }
  }
  // ---- selection of the lowest real parts ----
  if (t == 0) {
    int nsel = 0;
    // repeated minimum search (small k)
    for (int i = 0; i < m; ++i) vtmp[i] = 0.0;   // used flags
    while (nsel < want) {
      int best = -1;
      double bv = 0.0;
      for (int i = 0; i < m; ++i) {
        if (vtmp[i] != 0.0 || !(wr[i] < INFINITY)) continue;
        if (best < 0 || wr[i] < bv) {
          best = i;
          bv = wr[i];
        }
      }
      if (best < 0) break;
      vtmp[best] = 1.0;
      if (wi[best] != 0.0) {
        // mark the conjugate partner (adjacent from the 2 x 2 block)
        int partner = -1;
        if (best + 1 < m && wi[best + 1] == -wi[best] && wr[best + 1] == wr[best]) partner = best + 1;
        if (best > 0 && wi[best - 1] == -wi[best] && wr[best - 1] == wr[best]) partner = best - 1;
        if (partner >= 0) vtmp[partner] = 1.0;
        const int pos = wi[best] > 0.0 ? best : (partner >= 0 ? partner : best);
        sh.sel_idx[nsel] = pos;
        sh.sel_part[nsel] = 1;
        ++nsel;
        if (nsel < want) {
          sh.sel_idx[nsel] = pos;
          sh.sel_part[nsel] = 2;
          ++nsel;
        }
      } else {
        sh.sel_idx[nsel] = best;
        sh.sel_part[nsel] = 0;
        ++nsel;
      }
    }
    sh.iscal[2] = nsel;
    if (pb.mode == 1 && nsel > 0 && sh.sel_part[0] != 0) sh.iscal[1] = ST_COMPLEX;
  }
  __syncthreads();
  if (sh.iscal[1] != ST_OK) {
    if (t == 0) *pb.status = sh.iscal[1];
    return;
  }
  const int nsel = sh.iscal[2];
  // ---- 5./6. eigenvectors ----
  // W is free after each inverse iteration: W[0, m) and W[m, 2m) hold the back-transformed real
  // and imaginary parts.  A complex eigenvector is rotated so that its largest-magnitude
  // component is real and positive; its real part (kept alone when N_K ends inside the pair)
  // is then well defined.
  double* vr = W;
  double* vi = W + m;
  int last_idx = -1;
  for (int q = 0; q < nsel; ++q) {
    const int idx = sh.sel_idx[q];
    const int part = sh.sel_part[q];
    if (idx != last_idx) {
      hess_inverse_iteration(Hh, m, wr[idx], part ? wi[idx] : 0.0, anorm, W, yr, yi, plr, pli,
                             pswap, sh);
      for (int i = t; i < m; i += nt) {
        vr[i] = yr[i];
        vi[i] = yi[i];
      }
      __syncthreads();
      back_transform(A, hbeta, L, dsc, m, vr, sh);
      if (part) {
        back_transform(A, hbeta, L, dsc, m, vi, sh);
        if (t == 0) {
          int best = 0;
          double bv = -1.0;
          for (int i = 0; i < m; ++i) {
            const double a = vr[i] * vr[i] + vi[i] * vi[i];
            if (a > bv) {
              bv = a;
              best = i;
            }
          }
          const double nr = sqrt(bv);
          sh.scal[6] = vr[best] / nr;
          sh.scal[7] = vi[best] / nr;
        }
        __syncthreads();
        const double c = sh.scal[6], s = sh.scal[7];
        for (int i = t; i < m; i += nt) {
          const double a = vr[i], b = vi[i];
          vr[i] = a * c + b * s;       // (a + i b)(c - i s)
          vi[i] = b * c - a * s;
        }
        __syncthreads();
      }
      last_idx = idx;
    }
    double* out = pb.vec + (int64_t)q * m;
    const double* src = (part == 2) ? vi : vr;
    for (int i = t; i < m; i += nt) out[i] = src[i];
    if (t == 0) pb.lam[q] = wr[idx];
    __syncthreads();
  }
  if (t == 0) *pb.status = (nsel == (pb.mode == 1 ? 1 : pb.k)) ? ST_OK : ST_NOCONV;
}

__global__ void __launch_bounds__(kEigThreads)
eig_kernel(const EigProblem* __restrict__ probs) {
  extern __shared__ double dsm[];
  __shared__ Shared sh;
  dense_geig(probs[blockIdx.x], dsm, sh);
}

// ---------------------------------------------------------------------------------------------
// Generalized Davidson for the lowest eigenpair of H c = lambda S c (the combined problem of
// Eq. 7 when it is too large for the dense QR on one SM).  The basis V is kept S-orthonormal, so
// the projected problem V^T H V y = theta y is a small standard eigenproblem (solved with the
// dense routine above); the Ritz pair with the lowest real part is expanded with the diagonal
// preconditioner t = -(diag H - theta diag S)^-1 r, starting from the Psi direction e_0.
// Converged when ||H u - theta S u|| <= tol * ||S u|| * max(1, |theta|).
// ---------------------------------------------------------------------------------------------
constexpr int kDavMax = 40;

__device__ void matvec(const double* M, int m, const double* x, double* y) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = wid; i < m; i += nw) {
    const double* row = M + (int64_t)i * m;
    double s = 0.0;
    for (int j = lane; j < m; j += 32) s = fma(row[j], x[j], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[i] = s;
  }
  __syncthreads();
}

__device__ double dotv(const double* a, const double* b, int m, Shared& sh) {
  double p = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) p = fma(a[i], b[i], p);
  return block_sum(p, sh.red);
}

__global__ void __launch_bounds__(kEigThreads)
davidson_kernel(const EigProblem* __restrict__ probs, double tol, int max_iter) {
  extern __shared__ double dsm[];
  __shared__ Shared sh;
  __shared__ double hk[kDavMax * kDavMax];
  const EigProblem pb = probs[blockIdx.x];
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
  double* sLam = sW + (5 * ks * ks + 16 * ks);
  double* sVec = sLam + 2;
  int32_t* sStat = reinterpret_cast<int32_t*>(sVec + ks);

  for (int i = t; i < m; i += nt) {
    dH[i] = pb.H[(int64_t)i * m + i];
    dS[i] = pb.S[(int64_t)i * m + i];
  }
  __syncthreads();
  if (!(dS[0] > 0.0)) {
    if (t == 0) *pb.status = ST_NOT_PD;
    return;
  }
  // v_0 = e_0 / sqrt(S_00)
  for (int i = t; i < m; i += nt) V[i] = (i == 0) ? 1.0 / sqrt(dS[0]) : 0.0;
  __syncthreads();
  matvec(pb.H, m, V, HV);
  matvec(pb.S, m, V, SV);
  int k = 1;
  bool fresh = true;      // projected matrix must be rebuilt (start, restart)
  double theta = 0.0;
  int status = ST_NOCONV;
  for (int it = 0; it < max_iter; ++it) {
    // projected matrix: only the newest row and column change between restarts
    for (int i = 0; i < k; ++i) {
      const bool newer = (i == k - 1);
      for (int j = 0; j < k; ++j) {
        if (!fresh && !newer && j != k - 1) continue;
        const double v = dotv(V + (int64_t)i * m, HV + (int64_t)j * m, m, sh);
        if (t == 0) hk[i * kDavMax + j] = v;
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
    EigProblem sp{k, 1, 0, 0, sS, sH, sW, sLam, sVec, sStat};
    dense_geig(sp, dsm, sh);
    __syncthreads();
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
    if (rn <= tol * sn * fmax(1.0, fabs(theta))) {
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
    for (int pass = 0; pass < 2; ++pass)
      for (int j = 0; j < k; ++j) {
        const double c = dotv(SV + (int64_t)j * m, tv, m, sh);
        for (int i = t; i < m; i += nt) tv[i] -= c * V[(int64_t)j * m + i];
        __syncthreads();
      }
    double* stv = SV + (int64_t)k * m;
    matvec(pb.S, m, tv, stv);
    const double nn = dotv(tv, stv, m, sh);
    if (!(nn > 1e-300)) {
      status = ST_NOCONV;
      break;
    }
    const double inv = 1.0 / sqrt(nn);
    for (int i = t; i < m; i += nt) {
      tv[i] *= inv;
      stv[i] *= inv;
    }
    __syncthreads();
    matvec(pb.H, m, tv, HV + (int64_t)k * m);
    ++k;
  }
  if (t == 0) {
    *pb.status = status;
    pb.lam[0] = theta;
  }
  for (int i = t; i < m; i += nt) pb.vec[i] = u[i];
}

}  // namespace

size_t eig_work_doubles(int64_t m) {
  // 5 m^2 + 16 m for the dense solver; per-warp refinement storage (packed U, pivots),
  // candidate vectors and refined eigenvalues
  return (size_t)(5 * m * m + 16 * m + (int64_t)kRqiWarps * m * (m + 1) +
                  (int64_t)kRqiWarps * 3 * m + (int64_t)kMaxCand * 2 * m + 2 * kMaxCand + 64);
}

size_t davidson_work_doubles(int64_t m) {
  const int64_t ks = kDavMax;
  return (size_t)(3 * ks * m + 6 * m + 2 * ks * ks + 5 * ks * ks + 16 * ks + 2 + ks + 8);
}

void launch_davidson(const EigProblem* probs, int nprob, double tol, int max_iter,
                     cudaStream_t st) {
  if (nprob <= 0) return;
  const int smem = 200 * 1024;
  cudaFuncSetAttribute(davidson_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  davidson_kernel<<<nprob, kEigThreads, smem, st>>>(probs, tol, max_iter);
}

void launch_eig(const EigProblem* probs, int nprob, int threads, cudaStream_t st) {
  if (nprob <= 0) return;
  (void)threads;
  const int smem = 200 * 1024;
  cudaFuncSetAttribute(eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  eig_kernel<<<nprob, kEigThreads, smem, st>>>(probs);
}

}  // namespace blm
