// Sample sweeps on CUDA cores: reference shift, first-moment sums, tiled sample contractions
// and projections onto per-block directions.  These kernels form the plain FP64 path of the
// step (FP64 inputs) and the non-contraction parts of the mixed path (FP32 inputs).
//
// Eq. 3 (Sec. II.A): every matrix element is a weighted sum over samples of a product of two
// per-sample ratios; with the per-parameter reference shift c the sums are taken over
// O' = O - c and X' = E O' + G, and blm_assemble.cu turns them into centred matrices.
#include <cuda_runtime.h>
#include <stdint.h>

#include "blm_internal.cuh"

namespace blm {

namespace {

constexpr int kThreads = 256;

// ---------------------------------------------------------------------------------------------
// Column sums of O over a sample range (the first chunk's mean becomes the reference shift).
// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads)
colsum_kernel(const T* __restrict__ O, int64_t ns, int64_t ld, int64_t n, int64_t per_split,
              double* __restrict__ out) {
  const int64_t col = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (col >= n) return;
  const int64_t s0 = (int64_t)blockIdx.y * per_split;
  const int64_t s1 = min(ns, s0 + per_split);
  if (sizeof(T) == 4) {
    // FP32 samples: four double-float running sums (FP32 TwoSum, error term carried in a second
    // float), about 44 bits: the per-element FP64 conversion and add of a plain FP64 sum made
    // this pass FP64-pipe bound (2 FP64 operations per element, 3.9 ms per 65536 x 16384 chunk)
    float h[4] = {0.0f, 0.0f, 0.0f, 0.0f}, e[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    int64_t s = s0;
    for (; s + 3 < s1; s += 4) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float x = (float)O[(s + q) * ld + col];
        const float t = h[q] + x;
        const float bb = t - h[q];
        e[q] += (h[q] - (t - bb)) + (x - bb);
        h[q] = t;
      }
    }
    double acc = 0.0;
    for (; s < s1; ++s) acc += (double)O[s * ld + col];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc += (double)h[q] + (double)e[q];
    atomicAdd(out + col, acc);
  } else {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int64_t s = s0;
    for (; s + 3 < s1; s += 4) {
      a0 += (double)O[s * ld + col];
      a1 += (double)O[(s + 1) * ld + col];
      a2 += (double)O[(s + 2) * ld + col];
      a3 += (double)O[(s + 3) * ld + col];
    }
    for (; s < s1; ++s) a0 += (double)O[s * ld + col];
    atomicAdd(out + col, (a0 + a1) + (a2 + a3));
  }
}

// ---------------------------------------------------------------------------------------------
// First moments: sY += w (Y - shift), sEY += w E (Y - shift), sZ += w Z per column; and the
// scalars [sum w, sum w E] when scal != NULL.  FP32 inputs are summed in FP32 over runs of
// 32 samples and the run sums added in FP64 when A = float (the mixed path, whose O' is the
// FP32 value O - c); with A = double everything is FP64 (the FP64 path).
// ---------------------------------------------------------------------------------------------
template <typename T, typename A, typename TE = T>
__global__ void __launch_bounds__(kThreads)
sums_kernel(const T* __restrict__ Y, const T* __restrict__ Z, const TE* __restrict__ E,
            const TE* __restrict__ w, int64_t ns, int64_t ldy, int64_t ldz, int64_t ncols,
            int64_t per_split, const double* __restrict__ shift, double* __restrict__ sY,
            double* __restrict__ sEY, double* __restrict__ sZ, double* __restrict__ scal) {
  const int64_t col = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const int64_t s0 = (int64_t)blockIdx.y * per_split;
  const int64_t s1 = min(ns, s0 + per_split);
  if (scal != nullptr && blockIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int64_t s = s0 + threadIdx.x; s < s1; s += kThreads) {
      const double ws = w ? (double)w[s] : 1.0;
      a += ws;
      b += ws * (double)E[s];
    }
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(scal + 0, a);
      atomicAdd(scal + 1, b);
    }
  }
  if (col >= ncols) return;
  const A sh = shift ? (A)shift[col] : (A)0;
  double dY = 0.0, dEY = 0.0, dZ = 0.0;
  for (int64_t r = s0; r < s1; r += 32) {
    const int64_t re = min(s1, r + 32);
    A aY = 0, aEY = 0, aZ = 0;
    for (int64_t s = r; s < re; ++s) {
      const A ws = w ? (A)w[s] : (A)1;
      const A y = (A)Y[s * ldy + col] - sh;
      const A wy = ws * y;
      aY += wy;
      aEY += wy * (A)E[s];
      if (Z) aZ += ws * (A)Z[s * ldz + col];
    }
    dY += (double)aY;
    dEY += (double)aEY;
    dZ += (double)aZ;
  }
  atomicAdd(sY + col, dY);
  atomicAdd(sEY + col, dEY);
  if (Z) atomicAdd(sZ + col, dZ);
}

// ---------------------------------------------------------------------------------------------
// Tiled FP64 contraction over samples: out[i, j] += sum_s w_s A(s, i) B(s, j), 64 x 64 tiles,
// 16 samples per stage, 4 x 4 outputs per thread.  blockIdx.x = tile, blockIdx.y = sample split.
// ---------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ double seg_value(const Seg& sg, const SrcArgs<T>& a, int64_t s,
                                            int64_t c) {
  const int64_t col = sg.col0 + c;
  const int64_t idx = s * a.ld[sg.src] + col;
  double y = sg.src == 0 ? (double)a.Y0[idx] : a.Y1[idx];
  if (sg.src == 0 && a.shift) y -= a.shift[col];
  if (sg.xform) y = (double)a.E[s] * y + (sg.src == 0 ? (double)a.Z0[idx] : a.Z1[idx]);
  return y;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
contract_kernel(const Seg* __restrict__ segs, const Tile* __restrict__ tiles, SrcArgs<T> src,
                int64_t ns, int64_t per_split) {
  __shared__ double As[16][64];
  __shared__ double Bs[16][64];
  const Tile tl = tiles[blockIdx.x];
  const Seg sa = segs[tl.a_seg];
  const Seg sb = segs[tl.b_seg];
  const int64_t s0 = (int64_t)blockIdx.y * per_split;
  const int64_t s1 = min(ns, s0 + per_split);
  const int t = threadIdx.x;
  const int tx = t & 15, ty = t >> 4;
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;

  for (int64_t sb0 = s0; sb0 < s1; sb0 += 16) {
    for (int idx = t; idx < 16 * 64; idx += kThreads) {
      const int k = idx >> 6, c = idx & 63;
      const int64_t s = sb0 + k;
      double av = 0.0, bv = 0.0;
      if (s < s1) {
        if (c < tl.a_n) av = seg_value(sa, src, s, tl.a0 + c);
        if (c < tl.b_n) {
          bv = seg_value(sb, src, s, tl.b0 + c);
          if (src.w) bv *= (double)src.w[s];
        }
      }
      As[k][c] = av;
      Bs[k][c] = bv;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[k][ty * 4 + r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[k][tx * 4 + c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = ty * 4 + r;
    if (i >= tl.a_n) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = tx * 4 + c;
      if (j < tl.b_n) atomicAdd(tl.out + (int64_t)i * tl.out_ld + j, acc[r][c]);
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Projection onto per-block directions (Eq. 6 ratios p = Obar_b . B_j and r = G_b . B_j; the
// same kernel gives the history projections t = O'_k . D_jk, u = G_k . D_jk of Eq. 9).
// blockIdx.x = 32-sample tile, blockIdx.y = block; the block's parameters are taken in runs of
// 128 through shared memory.
// ---------------------------------------------------------------------------------------------
constexpr int kPS = 32;   // samples per CTA
constexpr int kPC = 128;  // parameters per shared-memory run
constexpr int kPL = kPC + 1;  // padded row: lanes reading different rows hit different banks

template <typename T, typename A, typename TO>
__global__ void __launch_bounds__(kThreads)
project_kernel(const T* __restrict__ O, const T* __restrict__ G, int64_t ldo, int64_t ldg,
               const double* __restrict__ shift, const ProjBlock* __restrict__ blocks,
               const double* __restrict__ cen, TO* __restrict__ Y, TO* __restrict__ Z,
               int64_t ldout, int64_t ns, int max_nd) {
  extern __shared__ unsigned char smem_raw[];
  A* Os = reinterpret_cast<A*>(smem_raw);          // kPS x kPL
  A* Gs = Os + kPS * kPL;                          // kPS x kPL
  A* Ds = Gs + kPS * kPL;                          // max_nd x kPL
  const ProjBlock pb = blocks[blockIdx.y];
  const int64_t s_base = (int64_t)blockIdx.x * kPS;
  const int t = threadIdx.x;
  const int npairs = kPS * pb.nd;                  // (sample, direction) pairs
  // up to 8 pairs per thread (kPS * max_nd <= 8 * kThreads is checked by the launcher)
  A accY[8], accZ[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) accY[q] = accZ[q] = (A)0;

  for (int p0 = 0; p0 < pb.m; p0 += kPC) {
    const int pc = min(kPC, pb.m - p0);
    for (int idx = t; idx < kPS * kPC; idx += kThreads) {
      const int k = idx / kPC, c = idx % kPC;
      const int64_t s = s_base + k;
      A ov = (A)0, gv = (A)0;
      if (s < ns && c < pc) {
        const int64_t col = pb.lo + p0 + c;
        ov = (A)O[s * ldo + col] - (shift ? (A)shift[col] : (A)0);
        gv = (A)G[s * ldg + col];
      }
      Os[k * kPL + c] = ov;
      Gs[k * kPL + c] = gv;
    }
    for (int idx = t; idx < pb.nd * kPC; idx += kThreads) {
      const int j = idx / kPC, c = idx % kPC;
      Ds[j * kPL + c] = (c < pc) ? (A)pb.dir[(int64_t)j * pb.dld + p0 + c] : (A)0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int pair = t + q * kThreads;
      if (pair < npairs) {
        const int k = pair / pb.nd, j = pair % pb.nd;
        const A* o = Os + k * kPL;
        const A* g = Gs + k * kPL;
        const A* d = Ds + j * kPL;
        A y = accY[q], z = accZ[q];
        for (int c = 0; c < pc; ++c) {
          y = fma(d[c], o[c], y);
          z = fma(d[c], g[c], z);
        }
        accY[q] = y;
        accZ[q] = z;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int pair = t + q * kThreads;
    if (pair < npairs) {
      const int k = pair / pb.nd, j = pair % pb.nd;
      const int64_t s = s_base + k;
      if (s < ns) {
        const int64_t oc = pb.oc + j;
        A y = accY[q];
        if (cen) y -= (A)cen[oc];
        Y[s * ldout + oc] = (TO)y;
        Z[s * ldout + oc] = (TO)accZ[q];
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Register-tiled projection (same results as project_kernel, for up to 32 directions).  A CTA
// takes 128 samples of one block; thread (sg, dg) owns samples 2 sg, 2 sg + 1 and directions
// DT dg .. DT dg + DT - 1 (DT = 5 for up to 20 directions, 8 for up to 32) of both
// Y = O'.B - cen and Z = G.B, so all 256 threads compute and each value read from shared memory
// feeds DT or two FMAs.  Runs of kC parameters are staged by cp.async, two stages in flight,
// small enough for two CTAs per SM; rows are padded to an odd length so that the eight sample
// rows a warp reads fall in different banks.
// ---------------------------------------------------------------------------------------------
constexpr int kTSp = 128;
template <typename A>
struct ProjCfg {
  static constexpr int kC = sizeof(A) == 4 ? 32 : 16;   // parameters per run
  static constexpr int kL = kC + 1;                     // padded row length
};

template <typename T, typename A>
constexpr size_t proj_tiled_smem() {
  return sizeof(T) * 2 * 2 * kTSp * ProjCfg<A>::kL + sizeof(A) * 2 * (32 * ProjCfg<A>::kL + ProjCfg<A>::kC);
}

template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int sz = valid ? (int)sizeof(T) : 0;   // 0: zero-fill
  if (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(sz) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(sz) : "memory");
}

template <typename T, typename A, typename TO, int DT>
__global__ void __launch_bounds__(kThreads, 2)
project_tiled_kernel(const T* __restrict__ O, const T* __restrict__ G, int64_t ldo, int64_t ldg,
                     const double* __restrict__ shift, const float* __restrict__ shift32,
                     const ProjBlock* __restrict__ blocks,
                     const double* __restrict__ cen, TO* __restrict__ Y, TO* __restrict__ Z,
                     int64_t ldout, int64_t ns) {
  constexpr int kC = ProjCfg<A>::kC, kL = ProjCfg<A>::kL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Os = reinterpret_cast<T*>(smem_raw);                    // [2][kTSp][kL]
  T* Gs = Os + 2 * kTSp * kL;                                 // [2][kTSp][kL]
  A* Ds = reinterpret_cast<A*>(Gs + 2 * kTSp * kL);           // [2][32][kL]
  A* Sh = Ds + 2 * 32 * kL;                                   // [2][kC]
  const ProjBlock pb = blocks[blockIdx.y];
  const int64_t s_base = (int64_t)blockIdx.x * kTSp;
  const int t = threadIdx.x;
  const int dgn = (pb.nd + DT - 1) / DT;                      // direction groups (<= 4)
  const bool active = t < (kTSp / 2) * dgn;
  const int sg = active ? t / dgn : 0, dg = active ? t % dgn : 0;
  const int nruns = (pb.m + kC - 1) / kC;

  auto issue = [&](int r) {
    const int st = r & 1;
    const int p0 = r * kC;
    const int pc = min(kC, pb.m - p0);
    T* os = Os + st * kTSp * kL;
    T* gs = Gs + st * kTSp * kL;
    for (int idx = t; idx < kTSp * kC; idx += kThreads) {
      const int k = idx / kC, c = idx - k * kC;
      const int64_t s = s_base + k;
      const bool ok = (s < ns) && (c < pc);
      const int64_t col = pb.lo + p0 + (c < pc ? c : 0);
      const int64_t srow = s < ns ? s : 0;
      cp_async_elem(os + k * kL + c, O + srow * ldo + col, ok);
      cp_async_elem(gs + k * kL + c, G + srow * ldg + col, ok);
    }
    // directions and shift in the accumulation type when memory holds them so (cp.async),
    // else converted on the way
    const A* dirA = nullptr;
    const A* shA = nullptr;
    if constexpr (sizeof(A) == 4) {
      dirA = reinterpret_cast<const A*>(pb.dir32);
      shA = reinterpret_cast<const A*>(shift32);
    } else {
      dirA = reinterpret_cast<const A*>(pb.dir);
      shA = reinterpret_cast<const A*>(shift);
    }
    A* ds = Ds + st * 32 * kL;
    for (int idx = t; idx < 32 * kC; idx += kThreads) {
      const int j = idx / kC, c = idx - j * kC;
      const bool ok = j < pb.nd && c < pc;
      const int64_t off = ok ? (int64_t)j * pb.dld + p0 + c : 0;
      if (dirA)
        cp_async_elem(ds + j * kL + c, dirA + off, ok);
      else
        ds[j * kL + c] = ok ? (A)pb.dir[off] : (A)0;
    }
    for (int c = t; c < kC; c += kThreads) {
      const bool ok = shift != nullptr && c < pc;
      const int64_t off = ok ? pb.lo + p0 + c : 0;
      if (shA)
        cp_async_elem(Sh + st * kC + c, shA + off, ok);
      else
        Sh[st * kC + c] = ok ? (A)shift[off] : (A)0;
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };

  A accY[2][DT], accZ[2][DT];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < DT; ++j) accY[i][j] = accZ[i][j] = (A)0;

  issue(0);
  for (int r = 0; r < nruns; ++r) {
    if (r + 1 < nruns) {
      issue(r + 1);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    if (active) {
      const int st = r & 1;
      const T* os = Os + st * kTSp * kL + (2 * sg) * kL;
      const T* gs = Gs + st * kTSp * kL + (2 * sg) * kL;
      const A* ds = Ds + st * 32 * kL + (DT * dg) * kL;
      const A* sh = Sh + st * kC;
      const int pc = min(kC, pb.m - r * kC);
#pragma unroll 4
      for (int c = 0; c < pc; ++c) {
        const A shc = sh[c];
        A o[2], g[2], d[DT];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          o[i] = (A)os[i * kL + c] - shc;
          g[i] = (A)gs[i * kL + c];
        }
#pragma unroll
        for (int j = 0; j < DT; ++j) d[j] = ds[j * kL + c];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int j = 0; j < DT; ++j) {
            accY[i][j] = fma(d[j], o[i], accY[i][j]);
            accZ[i][j] = fma(d[j], g[i], accZ[i][j]);
          }
      }
    }
    __syncthreads();
  }
  if (!active) return;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int64_t s = s_base + 2 * sg + i;
    if (s >= ns) continue;
#pragma unroll
    for (int j = 0; j < DT; ++j) {
      const int jj = DT * dg + j;
      if (jj >= pb.nd) continue;
      const int64_t oc = pb.oc + jj;
      A y = accY[i][j];
      if (cen) y -= (A)cen[oc];
      Y[s * ldout + oc] = (TO)y;
      Z[s * ldout + oc] = (TO)accZ[i][j];
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Register-blocked FP32 projection (mixed path; blocks of up to 20 directions whose parameter
// offsets and sample rows are 16-byte aligned).  A CTA of four warps takes 256 samples of one
// block: warps 0-1 form O' = O - c, warps 2-3 read G, and each lane owns four samples (rows
// lane + 32 s of its warp's 128) times all 20 directions, so a 16-byte shared load of four
// parameters of one sample feeds 80 products and every direction load is a broadcast.  The
// products use paired FP32 FMAs (fma.rn.f32x2: two independent round-to-nearest FMAs, bit for
// bit the scalar ones, so the sums equal project_tiled_kernel's).  Runs of 16 parameters are
// staged by 16-byte cp.async, double-buffered; sample rows are 64 bytes with their four
// 16-byte chunks XOR-swizzled by bits 1-2 of the row, so that the eight rows of a quarter-warp
// load, and the eight chunks of a quarter-warp's copies, fall in different bank groups.
// ---------------------------------------------------------------------------------------------
constexpr int kRbThreads = 128;
constexpr int kRbS = 256;       // samples per CTA
constexpr int kRbC = 16;        // parameters per stage
constexpr int kRbJ = 20;        // directions per thread
constexpr int kRbStages = 2;     // 68 KB: three CTAs (12 warps) per SM
constexpr int kRbTile = kRbS * kRbC;                       // floats of one O or G stage
constexpr int kRbStage = 2 * kRbTile + kRbC * kRbJ + kRbC;  // O, G, D [c][j], shift
constexpr size_t kRbSmem = sizeof(float) * kRbStages * kRbStage;

__device__ __forceinline__ int rb_swz(int r, int q) { return r * kRbC + ((q ^ ((r >> 1) & 3)) << 2); }

__device__ __forceinline__ void ffma2(unsigned long long& acc, unsigned long long a,
                                      unsigned long long b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(a), "l"(b));
}

__device__ __forceinline__ unsigned long long dup2(float x) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src, int bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(bytes)
               : "memory");
}

__global__ void __launch_bounds__(kRbThreads, 3)
project_rb_kernel(const float* __restrict__ O, const float* __restrict__ G, int64_t ld,
                  const float* __restrict__ shift32, const ProjBlock* __restrict__ blocks,
                  const double* __restrict__ cen, float* __restrict__ Y, float* __restrict__ Z,
                  int64_t ldout, int64_t ns) {
  extern __shared__ __align__(16) float rb_smem[];
  const ProjBlock pb = blocks[blockIdx.y];
  const int64_t s_base = (int64_t)blockIdx.x * kRbS;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const bool isO = warp < 2;
  const int nruns = (pb.m + kRbC - 1) / kRbC;

  auto issue = [&](int r) {
    if (r < nruns) {
      float* stg = rb_smem + (r % kRbStages) * kRbStage;
      const int p0 = r * kRbC;
      const int pc = min(kRbC, pb.m - p0);
#pragma unroll 4
      for (int idx = t; idx < 2 * kRbS * 4; idx += kRbThreads) {
        const int op = idx >> 10, i = idx & 1023, row = i >> 2, q = i & 3;
        const int64_t s = s_base + row;
        const int rem = (pc - 4 * q) * 4;
        const int bytes = s < ns ? (rem < 0 ? 0 : (rem > 16 ? 16 : rem)) : 0;
        const float* base = op ? G : O;
        const float* src = bytes ? base + s * ld + pb.lo + p0 + 4 * q : base;
        cp_async16(stg + op * kRbTile + rb_swz(row, q), src, bytes);
      }
      float* ds = stg + 2 * kRbTile;
      for (int idx = t; idx < kRbC * kRbJ; idx += kRbThreads) {
        const int c = idx / kRbJ, j = idx - c * kRbJ;
        const bool ok = j < pb.nd && c < pc;
        cp_async_elem(ds + idx, pb.dir32 + (ok ? (int64_t)j * pb.dld + p0 + c : 0), ok);
      }
      if (t < kRbC) {
        const bool ok = shift32 != nullptr && t < pc;
        cp_async_elem(ds + kRbC * kRbJ + t, ok ? shift32 + pb.lo + p0 + t : pb.dir32, ok);
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };

  unsigned long long acc[4][kRbJ / 2];
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int j = 0; j < kRbJ / 2; ++j) acc[s][j] = 0ull;

  const int rbase = (warp & 1) * 128 + lane;
  issue(0);
  for (int r = 0; r < nruns; ++r) {
    issue(r + 1);
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    __syncthreads();
    const float* stg = rb_smem + (r % kRbStages) * kRbStage;
    const float* tile = stg + (isO ? 0 : kRbTile);
    const float* ds = stg + 2 * kRbTile;
#pragma unroll
    for (int c4 = 0; c4 < kRbC / 4; ++c4) {
      float4 o[4];
#pragma unroll
      for (int s = 0; s < 4; ++s)
        o[s] = *reinterpret_cast<const float4*>(tile + rb_swz(rbase + 32 * s, c4));
      if (isO) {
        const float4 sh = *reinterpret_cast<const float4*>(ds + kRbC * kRbJ + 4 * c4);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          o[s].x -= sh.x; o[s].y -= sh.y; o[s].z -= sh.z; o[s].w -= sh.w;
        }
      }
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        unsigned long long od[4];
#pragma unroll
        for (int s = 0; s < 4; ++s)
          od[s] = dup2(cc == 0 ? o[s].x : cc == 1 ? o[s].y : cc == 2 ? o[s].z : o[s].w);
        const float* drow = ds + (4 * c4 + cc) * kRbJ;
#pragma unroll
        for (int jq = 0; jq < kRbJ / 4; ++jq) {
          const ulonglong2 dd = *reinterpret_cast<const ulonglong2*>(drow + 4 * jq);
#pragma unroll
          for (int s = 0; s < 4; ++s) {
            ffma2(acc[s][2 * jq], od[s], dd.x);
            ffma2(acc[s][2 * jq + 1], od[s], dd.y);
          }
        }
      }
    }
    __syncthreads();
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");

  float* out = isO ? Y : Z;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int64_t smp = s_base + rbase + 32 * s;
    if (smp >= ns) continue;
#pragma unroll
    for (int jp = 0; jp < kRbJ / 2; ++jp) {
      float v0, v1;
      asm("mov.b64 {%0, %1}, %2;" : "=f"(v0), "=f"(v1) : "l"(acc[s][jp]));
      const int j0 = 2 * jp;
      if (j0 < pb.nd) {
        const int64_t oc = pb.oc + j0;
        out[smp * ldout + oc] = (isO && cen) ? v0 - (float)cen[oc] : v0;
      }
      if (j0 + 1 < pb.nd) {
        const int64_t oc = pb.oc + j0 + 1;
        out[smp * ldout + oc] = (isO && cen) ? v1 - (float)cen[oc] : v1;
      }
    }
  }
}

int splits_for(int64_t ns, int64_t granule, int64_t max_splits) {
  int64_t s = (ns + granule - 1) / granule;
  if (s > max_splits) s = max_splits;
  if (s < 1) s = 1;
  return (int)s;
}

}  // namespace

template <typename T>
void launch_colmean(const T* O, int64_t ns, int64_t ld, int64_t n, double* sum_out,
                    cudaStream_t st) {
  if (ns <= 0) return;
  const int splits = splits_for(ns, 512, 256);
  const int64_t per = (ns + splits - 1) / splits;
  dim3 grid((unsigned)((n + kThreads - 1) / kThreads), (unsigned)splits);
  colsum_kernel<T><<<grid, kThreads, 0, st>>>(O, ns, ld, n, per, sum_out);
}

template <typename T>
void launch_sums(const T* Y, const T* Z, const T* E, const T* w, int64_t ns, int64_t ldy,
                 int64_t ldz, int64_t ncols, const double* shift, double* sY, double* sEY,
                 double* sZ, double* scal, bool fp32_runs, cudaStream_t st) {
  if (ns <= 0) return;
  const int64_t colblocks = (ncols + kThreads - 1) / kThreads;
  const int splits = splits_for(ns, 256, (int64_t)4 * 152 * 4 / (colblocks > 0 ? colblocks : 1) + 1);
  const int64_t per = ((ns + splits - 1) / splits + 31) / 32 * 32;
  dim3 grid((unsigned)(colblocks > 0 ? colblocks : 1), (unsigned)splits);
  if (fp32_runs)
    sums_kernel<T, float><<<grid, kThreads, 0, st>>>(Y, Z, E, w, ns, ldy, ldz, ncols, per, shift,
                                                     sY, sEY, sZ, scal);
  else
    sums_kernel<T, double><<<grid, kThreads, 0, st>>>(Y, Z, E, w, ns, ldy, ldz, ncols, per, shift,
                                                      sY, sEY, sZ, scal);
}

template <typename TE>
void launch_sums_mixed(const double* Y, const double* Z, const TE* E, const TE* w, int64_t ns,
                       int64_t ncols, double* sY, double* sEY, double* sZ, cudaStream_t st) {
  if (ns <= 0) return;
  const int64_t colblocks = (ncols + kThreads - 1) / kThreads;
  const int splits = splits_for(ns, 256, (int64_t)4 * 152 * 4 / (colblocks > 0 ? colblocks : 1) + 1);
  const int64_t per = ((ns + splits - 1) / splits + 31) / 32 * 32;
  dim3 grid((unsigned)(colblocks > 0 ? colblocks : 1), (unsigned)splits);
  sums_kernel<double, double, TE><<<grid, kThreads, 0, st>>>(Y, Z, E, w, ns, ncols, ncols, ncols,
                                                              per, nullptr, sY, sEY, sZ, nullptr);
}

template <typename T>
void launch_contract(const Seg* segs, const Tile* tiles, int ntiles, const SrcArgs<T>& src,
                     int64_t ns, int splits, cudaStream_t st) {
  if (ns <= 0 || ntiles <= 0) return;
  if (splits < 1) splits = 1;
  int64_t per = (ns + splits - 1) / splits;
  per = (per + 15) / 16 * 16;
  splits = (int)((ns + per - 1) / per);
  dim3 grid((unsigned)ntiles, (unsigned)splits);
  contract_kernel<T><<<grid, kThreads, 0, st>>>(segs, tiles, src, ns, per);
}

bool launch_project_rb(const float* O, const float* G, int64_t ld, const float* shift32,
                       const ProjBlock* blocks, int nblocks, bool offsets_aligned,
                       const double* cen, float* Y, float* Z, int64_t ldout, int64_t ns,
                       int max_nd, cudaStream_t st) {
  if (!offsets_aligned || max_nd > kRbJ || ld % 4 != 0 ||
      (((uintptr_t)O | (uintptr_t)G) & 15) != 0)
    return false;
  if (ns <= 0 || nblocks <= 0) return true;
  cudaFuncSetAttribute(project_rb_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)kRbSmem);
  dim3 grid((unsigned)((ns + kRbS - 1) / kRbS), (unsigned)nblocks);
  project_rb_kernel<<<grid, kRbThreads, kRbSmem, st>>>(O, G, ld, shift32, blocks, cen, Y, Z,
                                                       ldout, ns);
  return true;
}

template <typename T, typename TO>
void launch_project(const T* O, const T* G, int64_t ldo, int64_t ldg, const double* shift,
                    const float* shift32, const ProjBlock* blocks, int nblocks, const double* cen, TO* Y, TO* Z,
                    int64_t ldout, int64_t ns, int max_m, int max_nd, cudaStream_t st) {
  (void)max_m;
  if (ns <= 0 || nblocks <= 0) return;
  using A = TO;   // FP64 path: FP64 throughout; mixed path: FP32 products and sums
  if (max_nd <= 32) {
    constexpr size_t smem_t = proj_tiled_smem<T, A>();
    dim3 grid((unsigned)((ns + kTSp - 1) / kTSp), (unsigned)nblocks);
    if (max_nd <= 20) {
      cudaFuncSetAttribute(project_tiled_kernel<T, A, TO, 5>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_t);
      project_tiled_kernel<T, A, TO, 5><<<grid, kThreads, smem_t, st>>>(
          O, G, ldo, ldg, shift, shift32, blocks, cen, Y, Z, ldout, ns);
    } else {
      cudaFuncSetAttribute(project_tiled_kernel<T, A, TO, 8>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_t);
      project_tiled_kernel<T, A, TO, 8><<<grid, kThreads, smem_t, st>>>(
          O, G, ldo, ldg, shift, shift32, blocks, cen, Y, Z, ldout, ns);
    }
    return;
  }
  const size_t smem = sizeof(A) * (size_t)(2 * kPS * kPL + max_nd * kPL);
  cudaFuncSetAttribute(project_kernel<T, A, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem);
  dim3 grid((unsigned)((ns + kPS - 1) / kPS), (unsigned)nblocks);
  project_kernel<T, A, TO><<<grid, kThreads, smem, st>>>(O, G, ldo, ldg, shift, blocks, cen, Y, Z,
                                                         ldout, ns, max_nd);
}

__global__ void to_f32_kernel(const double* __restrict__ src, float* __restrict__ dst,
                              int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

void launch_to_f32(const double* src, float* dst, int64_t count, cudaStream_t st) {
  if (count <= 0) return;
  const int64_t blocks = (count + kThreads - 1) / kThreads;
  to_f32_kernel<<<(unsigned)(blocks < 1024 ? blocks : 1024), kThreads, 0, st>>>(src, dst, count);
}

template void launch_colmean<double>(const double*, int64_t, int64_t, int64_t, double*,
                                     cudaStream_t);
template void launch_colmean<float>(const float*, int64_t, int64_t, int64_t, double*,
                                    cudaStream_t);
template void launch_sums<double>(const double*, const double*, const double*, const double*,
                                  int64_t, int64_t, int64_t, int64_t, const double*, double*,
                                  double*, double*, double*, bool, cudaStream_t);
template void launch_sums<float>(const float*, const float*, const float*, const float*, int64_t,
                                 int64_t, int64_t, int64_t, const double*, double*, double*,
                                 double*, double*, bool, cudaStream_t);
template void launch_project<double, double>(const double*, const double*, int64_t, int64_t,
                                             const double*, const float*, const ProjBlock*, int, const double*,
                                             double*, double*, int64_t, int64_t, int, int,
                                             cudaStream_t);
template void launch_project<float, float>(const float*, const float*, int64_t, int64_t,
                                           const double*, const float*, const ProjBlock*, int, const double*,
                                           float*, float*, int64_t, int64_t, int, int,
                                           cudaStream_t);
template void launch_project<float, double>(const float*, const float*, int64_t, int64_t,
                                            const double*, const float*, const ProjBlock*, int, const double*,
                                            double*, double*, int64_t, int64_t, int, int,
                                            cudaStream_t);
template void launch_sums_mixed<double>(const double*, const double*, const double*,
                                        const double*, int64_t, int64_t, double*, double*,
                                        double*, cudaStream_t);
template void launch_sums_mixed<float>(const double*, const double*, const float*, const float*,
                                       int64_t, int64_t, double*, double*, double*, cudaStream_t);
template void launch_contract<double>(const Seg*, const Tile*, int, const SrcArgs<double>&,
                                      int64_t, int, cudaStream_t);
template void launch_contract<float>(const Seg*, const Tile*, int, const SrcArgs<float>&,
                                     int64_t, int, cudaStream_t);

}  // namespace blm
