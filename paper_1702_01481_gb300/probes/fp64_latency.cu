// FP64 / FP32 latency and throughput on one SM, and barrier cost, measured with clock64.
// Build and run: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o /tmp/fp64_latency \
//   paper_1702_01481_gb300/probes/fp64_latency.cu && /tmp/fp64_latency
#include <cstdio>
#include <cuda_runtime.h>
__global__ void probe(double a, double b, long long* out, double* sink, int mode, int n) {
  const int t = threadIdx.x;
  double x = a + t * 1e-9, y = b, x2 = x + 1, x3 = x + 2, x4 = x + 3, x5 = x + 4, x6 = x + 5, x7 = x + 6, x8 = x + 7;
  __syncthreads();
  long long c0 = clock64();
  if (mode == 0) {              // dependent FMA, lane 0 only
    if (t == 0) for (int i = 0; i < n; ++i) x = fma(x, a, b);
  } else if (mode == 1) {       // dependent FMA, all lanes of warp 0
    if (t < 32) for (int i = 0; i < n; ++i) x = fma(x, a, b);
  } else if (mode == 2) {       // 8 chains, warp 0
    if (t < 32) for (int i = 0; i < n; ++i) { x = fma(x, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b); x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b); x8 = fma(x8, a, b); }
  } else if (mode == 3) {       // 8 chains, all threads of the block
    for (int i = 0; i < n; ++i) { x = fma(x, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b); x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b); x8 = fma(x8, a, b); }
  } else if (mode == 4) {       // dependent division, lane 0
    if (t == 0) for (int i = 0; i < n; ++i) x = b / x + a;
  } else if (mode == 5) {       // dependent division, warp 0
    if (t < 32) for (int i = 0; i < n; ++i) x = b / x + a;
  } else if (mode == 6) {       // dependent sqrt, lane 0
    if (t == 0) for (int i = 0; i < n; ++i) x = sqrt(x) + a;
  } else if (mode == 7) {       // barrier
    for (int i = 0; i < n; ++i) __syncthreads();
  } else if (mode == 8) {       // named barrier over the first 128 threads
    if (t < 128) for (int i = 0; i < n; ++i) asm volatile("bar.sync 1, 128;");
  } else if (mode == 9) {       // dependent FP32 FMA lane 0
    float xf = (float)x;
    if (t == 0) for (int i = 0; i < n; ++i) xf = fmaf(xf, (float)a, (float)b);
    x = xf;
  } else if (mode == 10) {      // 8 chains, one warp per SMSP (threads 0..127, warps 0..3)
    if (t < 128) for (int i = 0; i < n; ++i) { x = fma(x, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b); x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b); x8 = fma(x8, a, b); }
  } else if (mode == 11) {      // dependent FMA, 8 lanes of warp 0
    if (t < 8) for (int i = 0; i < n; ++i) x = fma(x, a, b);
  }
  __syncthreads();
  long long c1 = clock64();
  if (t == 0) out[0] = c1 - c0;
  sink[t] = x + x2 + x3 + x4 + x5 + x6 + x7 + x8 + y;
}
int main() {
  long long* d; double* s; cudaMalloc(&d, 8); cudaMalloc(&s, 1024 * 8);
  const char* names[] = {"fma dep lane0", "fma dep warp", "fma 8ch warp", "fma 8ch block", "div dep lane0", "div dep warp", "sqrt dep lane0", "syncthreads", "bar.sync 128", "f32 fma dep lane0", "fma 8ch 4warps", "fma dep 8 lanes"};
  int threads[] = {128, 512};
  for (int th : threads)
    for (int mode = 0; mode < 12; ++mode) {
      const int n = 4096;
      long long best = 1LL << 62;
      for (int r = 0; r < 3; ++r) {
        probe<<<1, th>>>(0.999999, 1e-7, d, s, mode, n);
        long long h; cudaMemcpy(&h, d, 8, cudaMemcpyDeviceToHost);
        if (h < best) best = h;
      }
      cudaError_t e = cudaDeviceSynchronize();
      printf("threads %4d  %-20s  %8.2f cycles per iteration (%s)\n", th, names[mode], (double)best / n, cudaGetErrorString(e));
    }
  return 0;
}
