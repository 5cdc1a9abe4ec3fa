// FP64 assembly of the eigenproblem matrices from the sweep sums (Eq. 3 in the centred basis).
//
// The sweeps accumulate raw sums over shifted ratios a' = a - c (c: the reference shift) and the
// X-type ratios y' of the Hamiltonian side.  With <.> = sum_s w_s (.) / sum_s w_s, the centred
// matrices follow exactly from
//   S[a][c] = <a' c'> - <a'><c'>
//   H[a][c] = <a' y'_c> - <a'><y'_c> - mu_c (<a' E> - <a'><E>)        (mu_c = <c'>)
//   H[0][c] = <y'_c> - mu_c <E>,   H[a][0] = <a' E> - <a'><E>,   H[0][0] = <E>,
//   S[0][0] = 1,  S[0][c] = S[a][0] = 0,
// because the centred ratio of the Hamiltonian side is y'_c - mu_c E (X = E Obar + G).
// The diagonal shift of Sec. II.A enters as shift * (Gram matrix of the basis directions).
#include <cuda_runtime.h>
#include <stdint.h>

#include "blm_internal.cuh"

namespace blm {

namespace {

struct Terms {
  double mean;    // <a'>
  double meanE;   // <a' E>
  double ymean;   // <y'_a>  (Hamiltonian-side ratio of the same direction)
};

// Block b's tangent index a -> parameter (a < m) or history column r (virtual column r = k N_O + j
// for direction j of block k; the block's basis lists them j-major, k ascending, k != b).
__device__ __forceinline__ void hist_index(int h, int b, int n_old, int n_blocks, int& r) {
  const int per = n_blocks - 1;
  const int j = h / per;
  int k = h % per;
  if (k >= b) ++k;
  r = k * n_old + j;
  (void)n_old;
}

__global__ void assemble_blocks_kernel(const BlockAsm* __restrict__ blocks, const double* sO,
                                       const double* sEO, const double* sG,
                                       const double* scal, HistSums hist, double shift) {
  const BlockAsm ba = blocks[blockIdx.y];
  const int D = ba.d + 1;
  const int64_t total = (int64_t)D * D;
  const double sw = scal[0];
  const double iw = 1.0 / sw;
  const double Em = scal[1] * iw;
  const int m = ba.m;
  const int R = hist.n_old * hist.n_blocks;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int ai = (int)(idx / D), ci = (int)(idx % D);
    double s = 0.0, hv = 0.0;
    if (ai == 0 && ci == 0) {
      s = 1.0;
      hv = Em;
    } else {
      // terms of the row direction a and column direction c
      Terms ta{0, 0, 0}, tc{0, 0, 0};
      int ra = -1, rc = -1;
      const int a = ai - 1, c = ci - 1;
      if (ai > 0) {
        if (a < m) {
          const int64_t p = ba.lo + a;
          ta = Terms{sO[p] * iw, sEO[p] * iw, (sEO[p] + sG[p]) * iw};
        } else {
          hist_index(a - m, ba.b, hist.n_old, hist.n_blocks, ra);
          ta = Terms{hist.sT[ra] * iw, hist.sET[ra] * iw, (hist.sET[ra] + hist.sU[ra]) * iw};
        }
      }
      if (ci > 0) {
        if (c < m) {
          const int64_t p = ba.lo + c;
          tc = Terms{sO[p] * iw, sEO[p] * iw, (sEO[p] + sG[p]) * iw};
        } else {
          hist_index(c - m, ba.b, hist.n_old, hist.n_blocks, rc);
          tc = Terms{hist.sT[rc] * iw, hist.sET[rc] * iw, (hist.sET[rc] + hist.sU[rc]) * iw};
        }
      }
      if (ai == 0) {
        s = 0.0;
        hv = tc.ymean - tc.mean * Em;
      } else if (ci == 0) {
        s = 0.0;
        hv = ta.meanE - ta.mean * Em;
      } else {
        // raw second moments <a' c'> (both orders, for symmetry) and <a' y'_c>
        double ac, ca, ay;
        if (a < m && c < m) {
          ac = ba.C[(int64_t)a * 2 * m + c] * iw;
          ca = ba.C[(int64_t)c * 2 * m + a] * iw;
          ay = ba.C[(int64_t)a * 2 * m + m + c] * iw;
        } else if (a < m) {   // parameter row, history column
          const int64_t p = ba.lo + a;
          ac = ca = hist.OT[p * 2 * R + rc] * iw;
          ay = hist.OT[p * 2 * R + R + rc] * iw;
        } else if (c < m) {   // history row, parameter column
          const int64_t p = ba.lo + c;
          ac = ca = hist.OT[p * 2 * R + ra] * iw;
          ay = hist.XT[p * R + ra] * iw;
        } else {
          ac = hist.TT[(int64_t)ra * 2 * R + rc] * iw;
          ca = hist.TT[(int64_t)rc * 2 * R + ra] * iw;
          ay = hist.TT[(int64_t)ra * 2 * R + R + rc] * iw;
        }
        s = 0.5 * (ac + ca) - ta.mean * tc.mean;
        hv = ay - ta.mean * tc.ymean - tc.mean * (ta.meanE - ta.mean * Em);
        if (shift != 0.0) {
          double g = 0.0;
          if (a < m && c < m) g = (a == c) ? 1.0 : 0.0;
          else if (a >= m && c >= m) g = hist.gram[(int64_t)ra * R + rc];
          hv += shift * g;
        }
      }
    }
    ba.S[idx] = s;
    ba.H[idx] = hv;
  }
}

__global__ void assemble_combined_kernel(int64_t dc, const double* C, const double* sY,
                                         const double* sEY, const double* sZ, const double* scal,
                                         const double* gram, double shift, double* S, double* H) {
  const int64_t D = dc + 1;
  const double iw = 1.0 / scal[0];
  const double Em = scal[1] * iw;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < D * D;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ai = idx / D, ci = idx % D;
    double s = 0.0, hv = 0.0;
    if (ai == 0 && ci == 0) {
      s = 1.0;
      hv = Em;
    } else if (ai == 0) {
      const int64_t c = ci - 1;
      const double mc = sY[c] * iw, yc = (sEY[c] + sZ[c]) * iw;
      hv = yc - mc * Em;
    } else if (ci == 0) {
      const int64_t a = ai - 1;
      hv = sEY[a] * iw - sY[a] * iw * Em;
    } else {
      const int64_t a = ai - 1, c = ci - 1;
      const double ma = sY[a] * iw, mc = sY[c] * iw;
      const double maE = sEY[a] * iw, yc = (sEY[c] + sZ[c]) * iw;
      // upper triangle only (the tensor-core path does not compute overlap tiles wholly below
      // the diagonal)
      const double su = (a <= c ? C[a * 2 * dc + c] : C[c * 2 * dc + a]) * iw;
      const double ay = C[a * 2 * dc + dc + c] * iw;
      s = su - ma * mc;
      hv = ay - ma * yc - mc * (maE - ma * Em);
      if (shift != 0.0 && gram) hv += shift * gram[a * dc + c];
    }
    S[idx] = s;
    H[idx] = hv;
  }
}

}  // namespace

void launch_assemble_blocks(const BlockAsm* blocks, int nblocks, int max_dim, const double* sO,
                            const double* sEO, const double* sG, const double* scal,
                            HistSums hist, double shift, cudaStream_t st) {
  const int64_t D = max_dim + 1;
  int gx = (int)((D * D + 255) / 256);
  if (gx > 1024) gx = 1024;
  dim3 grid(gx, nblocks);
  assemble_blocks_kernel<<<grid, 256, 0, st>>>(blocks, sO, sEO, sG, scal, hist, shift);
}

void launch_assemble_combined(int64_t dc, const double* C, const double* sY, const double* sEY,
                              const double* sZ, const double* scal, const double* gram,
                              double shift, double* S, double* H, cudaStream_t st) {
  const int64_t D = dc + 1;
  int gx = (int)((D * D + 255) / 256);
  if (gx > 4096) gx = 4096;
  assemble_combined_kernel<<<gx, 256, 0, st>>>(dc, C, sY, sEY, sZ, scal, gram, shift, S, H);
}

}  // namespace blm
