// Small FP64 kernels around the solves: retained directions B^(b) from the block eigenvectors
// (Sec. II.B), their centring constants and Gram matrices, and the update of Eq. 8.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "blm_internal.cuh"

namespace blm {

namespace {

__device__ double cta_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  __syncthreads();
  return s;
}

// B^(b) row q = beta part of eigenvector q (components 1 .. M_b), unit 2-norm, largest-magnitude
// entry positive.  One CTA per block.
__global__ void extract_dirs_kernel(const DirBlock* __restrict__ blocks) {
  __shared__ double red[32];
  __shared__ double smax[2];
  const DirBlock db = blocks[blockIdx.x];
  for (int q = 0; q < db.k; ++q) {
    const double* v = db.vec + (int64_t)q * db.d1 + 1;
    double part = 0.0;
    for (int i = threadIdx.x; i < db.m; i += blockDim.x) part += v[i] * v[i];
    const double nrm2 = cta_sum(part, red);
    if (threadIdx.x == 0) {
      int best = 0;
      double bv = -1.0;
      for (int i = 0; i < db.m; ++i)
        if (fabs(v[i]) > bv) {
          bv = fabs(v[i]);
          best = i;
        }
      smax[0] = v[best] < 0.0 ? -1.0 : 1.0;
      if (!(nrm2 > 0.0) || !isfinite(nrm2)) *db.status = ST_ZERO_DIR;
    }
    __syncthreads();
    const double sc = (nrm2 > 0.0) ? smax[0] / sqrt(nrm2) : 0.0;
    for (int i = threadIdx.x; i < db.m; i += blockDim.x) db.B[(int64_t)q * db.m + i] = v[i] * sc;
    __syncthreads();
  }
}

// cen[oc + j] = dir_j . m'_b  with m' = sO / sum w (the shifted mean), so that the projected
// ratio dir_j . (O - c) - cen is centred.
__global__ void cen_kernel(const ProjBlock* __restrict__ blocks, const double* sO,
                           const double* scal, double* cen) {
  __shared__ double red[32];
  const ProjBlock pb = blocks[blockIdx.x];
  const double iw = 1.0 / scal[0];
  for (int j = 0; j < pb.nd; ++j) {
    double part = 0.0;
    for (int i = threadIdx.x; i < pb.m; i += blockDim.x)
      part += pb.dir[(int64_t)j * pb.dld + i] * sO[pb.lo + i] * iw;
    const double s = cta_sum(part, red);
    if (threadIdx.x == 0) cen[pb.oc + j] = s;
  }
}

// gram[oc + j, oc + j'] = dir_j . dir_j' within each block (zero across blocks: set by memset).
__global__ void gram_kernel(const ProjBlock* __restrict__ blocks, double* gram, int64_t ld) {
  __shared__ double red[32];
  const ProjBlock pb = blocks[blockIdx.x];
  for (int j = 0; j < pb.nd; ++j)
    for (int jj = 0; jj < pb.nd; ++jj) {
      double part = 0.0;
      for (int i = threadIdx.x; i < pb.m; i += blockDim.x)
        part += pb.dir[(int64_t)j * pb.dld + i] * pb.dir[(int64_t)jj * pb.dld + i];
      const double s = cta_sum(part, red);
      if (threadIdx.x == 0) gram[(int64_t)(pb.oc + j) * ld + pb.oc + jj] = s;
    }
}

// alpha = c_0 - sum_bj A_bj (B^(b)_j . m_b), m = c_shift + m' the sample mean of O (Eq. 8 with
// the centred basis converted back to the raw Psi coefficient).  One CTA.
__global__ void alpha_kernel(int nblocks, const ProjBlock* __restrict__ blocks, int64_t dc,
                             const double* c, const double* shift, const double* sO,
                             const double* scal, double* alpha, int32_t* status) {
  __shared__ double red[32];
  const double iw = 1.0 / scal[0];
  double part = 0.0, nrm = 0.0;
  for (int b = 0; b < nblocks; ++b) {
    const ProjBlock pb = blocks[b];
    for (int j = 0; j < pb.nd; ++j) {
      const double A = c[1 + pb.oc + j];
      for (int i = threadIdx.x; i < pb.m; i += blockDim.x) {
        const int64_t p = pb.lo + i;
        const double mean = shift[p] + sO[p] * iw;
        part += A * pb.dir[(int64_t)j * pb.dld + i] * mean;
      }
    }
  }
  for (int64_t q = threadIdx.x; q < dc + 1; q += blockDim.x) nrm += c[q] * c[q];
  const double s = cta_sum(part, red);
  const double n2 = cta_sum(nrm, red);
  if (threadIdx.x == 0) {
    const double a = c[0] - s;
    *alpha = a;
    if (!(fabs(a) > 1e-12 * sqrt(n2))) *status = ST_ALPHA;
  }
}

// dmu_{i in b} = sum_j A_bj B^(b)_ji / alpha (Eq. 8).  One CTA per block.
__global__ void dmu_kernel(const ProjBlock* __restrict__ blocks, const double* c,
                           const double* alpha, double* dmu) {
  const ProjBlock pb = blocks[blockIdx.x];
  const double ia = 1.0 / *alpha;
  for (int i = threadIdx.x; i < pb.m; i += blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < pb.nd; ++j) s += c[1 + pb.oc + j] * pb.dir[(int64_t)j * pb.dld + i];
    dmu[pb.lo + i] = s * ia;
  }
}

}  // namespace

void launch_extract_dirs(const DirBlock* blocks, int nblocks, cudaStream_t st) {
  if (nblocks > 0) extract_dirs_kernel<<<nblocks, 256, 0, st>>>(blocks);
}

void launch_cen(const ProjBlock* blocks, int nblocks, const double* sO, const double* scal,
                double* cen, cudaStream_t st) {
  if (nblocks > 0) cen_kernel<<<nblocks, 256, 0, st>>>(blocks, sO, scal, cen);
}

void launch_gram(const ProjBlock* blocks, int nblocks, int max_nd, double* gram, int64_t ld,
                 cudaStream_t st) {
  (void)max_nd;
  if (nblocks > 0) gram_kernel<<<nblocks, 256, 0, st>>>(blocks, gram, ld);
}

void launch_update(int nblocks, const ProjBlock* blocks, int64_t dc, const double* c,
                   const double* shift, const double* sO, const double* scal, double* alpha,
                   double* dmu, int32_t* status, cudaStream_t st) {
  alpha_kernel<<<1, 512, 0, st>>>(nblocks, blocks, dc, c, shift, sO, scal, alpha, status);
  dmu_kernel<<<nblocks, 256, 0, st>>>(blocks, c, alpha, dmu);
}

}  // namespace blm
