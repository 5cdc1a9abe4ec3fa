// Device twin of synth/workload.py: fills device buffers with the same seeded samples
//   O_s = Q (sigma * z_s),  E_s = -1 + O_s . g + 0.01 eps_s,
//   G_s = Q (diag(mu) Q^T O_s + 0.01 sigma * eta_s)
// using Philox4x32-10 (Salmon et al., SC'11) keyed by (seed, opt) with counter (idx_lo, idx_hi,
// tag, 0) and Box-Muller normals, exactly as the host module defines them.  Q = H_0 H_1 H_2 H_3
// with H_r = I - 2 u_r u_r^T; u, sigma, g, mu come from the host module (synth.make_model).
// Holds no arithmetic of the blocked linear method.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace {

constexpr int kThreads = 512;
constexpr uint32_t TAG_Z = 4, TAG_EPS = 5, TAG_ETA = 9;

struct U4 {
  uint32_t x0, x1, x2, x3;
};

__device__ __forceinline__ U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                     uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return U4{c0, c1, c2, c3};
}

__device__ __forceinline__ double u53(uint32_t a, uint32_t b) {
  return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6) + 0.5) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ double normal(uint64_t seed, uint64_t opt, uint32_t tag, uint64_t idx) {
  const U4 x = philox((uint32_t)idx, (uint32_t)(idx >> 32), tag, 0u, (uint32_t)seed, (uint32_t)opt);
  const double u1 = u53(x.x0, x.x1), u2 = u53(x.x2, x.x3);
  return sqrt(-2.0 * log(u1)) * cos(2.0 * 3.141592653589793 * u2);
}

__device__ double cta_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < kThreads / 32; ++i) s += red[i];
  __syncthreads();
  return s;
}

// v <- H_r v for r in `order`
__device__ void reflect(double* v, const double* u, int64_t n, int r, double* red) {
  const double* ur = u + (int64_t)r * n;
  double part = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += kThreads) part += v[i] * ur[i];
  const double d = 2.0 * cta_sum(part, red);
  for (int64_t i = threadIdx.x; i < n; i += kThreads) v[i] -= d * ur[i];
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
samples_kernel(int64_t n, int64_t s0, int64_t count, uint64_t seed, uint64_t opt, int noise,
               double offset, const double* __restrict__ u, const double* __restrict__ sigma,
               const double* __restrict__ g, const double* __restrict__ mu, T* __restrict__ O,
               T* __restrict__ G, T* __restrict__ E, int64_t ld) {
  extern __shared__ double v[];
  __shared__ double red[32];
  for (int64_t q = blockIdx.x; q < count; q += gridDim.x) {
    const int64_t s = s0 + q;
    for (int64_t i = threadIdx.x; i < n; i += kThreads)
      v[i] = normal(seed, opt, TAG_Z, (uint64_t)s * (uint64_t)n + (uint64_t)i) * sigma[i];
    __syncthreads();
    for (int r = 3; r >= 0; --r) reflect(v, u, n, r, red);   // O = H_0 H_1 H_2 H_3 (sigma z)
    double part = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += kThreads) {
      part += v[i] * g[i];
      O[q * ld + i] = (T)(v[i] + offset);
    }
    const double og = cta_sum(part, red);
    if (threadIdx.x == 0) {
      double eps;
      if (noise == 0) {
        eps = normal(seed, opt, TAG_EPS, (uint64_t)s);
      } else {
        const double z0 = normal(seed, opt, TAG_EPS, (uint64_t)s);
        double chi = 0.0;
        for (uint32_t k = 1; k <= 3; ++k) {
          const double zk = normal(seed, opt, TAG_EPS + k, (uint64_t)s);
          chi += zk * zk;
        }
        eps = z0 / sqrt(chi / 3.0);
      }
      E[q] = (T)(-1.0 + og + 0.01 * eps);
    }
    for (int r = 0; r < 4; ++r) reflect(v, u, n, r, red);    // Q^T O
    for (int64_t i = threadIdx.x; i < n; i += kThreads)
      v[i] = v[i] * mu[i] +
             0.01 * sigma[i] * normal(seed, opt, TAG_ETA, (uint64_t)s * (uint64_t)n + (uint64_t)i);
    __syncthreads();
    for (int r = 3; r >= 0; --r) reflect(v, u, n, r, red);   // Q (diag(mu) Q^T O + noise)
    for (int64_t i = threadIdx.x; i < n; i += kThreads) G[q * ld + i] = (T)v[i];
    __syncthreads();
  }
}

}  // namespace

extern "C" {

// Samples s0 .. s0+count-1 of optimisation (seed, opt) into device arrays O, G (count x ld) and
// E (count); out_f32 selects float outputs (the double draws rounded once).  u: 4 x n, sigma, g,
// mu: n, all device FP64.  Returns a cudaError_t value (0 = success).
int blmsynth_samples(int64_t n, int64_t s0, int64_t count, uint64_t seed, uint64_t opt,
                     int noise, double offset, const double* u, const double* sigma,
                     const double* g, const double* mu, void* O, void* G, void* E, int out_f32,
                     int64_t ld, void* stream) {
  if (count <= 0) return 0;
  const size_t smem = sizeof(double) * (size_t)n;
  if (smem > 200 * 1024) return (int)cudaErrorInvalidValue;
  cudaStream_t st = (cudaStream_t)stream;
  const int grid = (int)(count < 152 * 8 ? count : 152 * 8);
  if (out_f32) {
    cudaFuncSetAttribute(samples_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    samples_kernel<float><<<grid, kThreads, smem, st>>>(n, s0, count, seed, opt, noise, offset, u,
                                                        sigma, g, mu, (float*)O, (float*)G,
                                                        (float*)E, ld);
  } else {
    cudaFuncSetAttribute(samples_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    samples_kernel<double><<<grid, kThreads, smem, st>>>(n, s0, count, seed, opt, noise, offset,
                                                         u, sigma, g, mu, (double*)O, (double*)G,
                                                         (double*)E, ld);
  }
  return (int)cudaGetLastError();
}

}  // extern "C"
