// Internal declarations shared by the library's translation units (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/blm.h"

namespace blm {

// ---------------------------------------------------------------------------------------------
// Operand segments of the sample contractions.  A segment is a run of columns of one of two
// sample-major sources (src 0: the caller's sample arrays O, G; src 1: the handle's projection
// scratch Y, Z).  Its value for sample s, column c is
//   plain:  Y[s, col0 + c] - shift[col0 + c]
//   xform:  E[s] * (Y[s, col0 + c] - shift[col0 + c]) + Z[s, col0 + c]
// which are the ratios <n|Psibar^x>/<n|Psi> (up to the constant shift) and <n|H Psibar^x>/<n|Psi>
// of Eq. 3 when Y = O, Z = dE_L/dmu.  The shift applies to src 0 only.
// ---------------------------------------------------------------------------------------------
struct Seg {
  int32_t src;
  int32_t xform;
  int64_t col0;
};

// Source 0 holds the caller's samples (element type T: FP64, or FP32 widened to FP64 on load);
// source 1 is FP64 scratch.  E and w are the caller's (type T).
template <typename T>
struct SrcArgs {
  const T* Y0;
  const double* Y1;
  const T* Z0;
  const double* Z1;
  int64_t ld[2];
  const double* shift;
  const T* E;
  const T* w;
};

// One 64 x 64 output tile: C[a0 + i, b0 + j] += sum_s w_s A(s, a0 + i) B(s, b0 + j),
// i < a_n, j < b_n, A from segment a_seg, B from segment b_seg; out points at C[a0, b0].
struct Tile {
  int32_t a_seg, b_seg;
  int32_t a0, b0;
  int32_t a_n, b_n;
  int32_t pad0, pad1;
  double* out;
  int64_t out_ld;
};

// Projection of every sample onto per-block directions:
//   Y[s, oc + j] = sum_i dir[j, i] (O[s, lo + i] - shift[lo + i]) - cen[oc + j]
//   Z[s, oc + j] = sum_i dir[j, i] G[s, lo + i]
struct ProjBlock {
  int64_t lo;        // first parameter of the block
  int32_t m;         // parameters in the block
  int32_t nd;        // directions
  int32_t oc;        // first output column
  int32_t pad;
  const double* dir; // nd rows of m values, row stride dld
  int64_t dld;
  const float* dir32;  // the same rows in FP32 (mixed path), or nullptr
};

enum { ST_OK = 0, ST_NOT_PD = 1, ST_NONFINITE = 2, ST_COMPLEX = 3, ST_NOCONV = 4, ST_ALPHA = 5,
       ST_ZERO_DIR = 6 };

// ------------------------------- launchers (blm_sweep_f64.cu) --------------------------------
template <typename T>
void launch_colmean(const T* O, int64_t ns, int64_t ld, int64_t n, double* sum_out,
                    cudaStream_t st);
template <typename T>
void launch_sums(const T* Y, const T* Z, const T* E, const T* w, int64_t ns, int64_t ldy,
                 int64_t ldz, int64_t ncols, const double* shift, double* sY, double* sEY,
                 double* sZ, double* scal /* [sw, sE] or NULL */, bool fp32_runs,
                 cudaStream_t st);
// First moments of FP64 scratch columns (projections) with the caller's E and w (type TE):
// sY += w Y, sEY += w E Y, sZ += w Z.
template <typename TE>
void launch_sums_mixed(const double* Y, const double* Z, const TE* E, const TE* w, int64_t ns,
                       int64_t ncols, double* sY, double* sEY, double* sZ, cudaStream_t st);
template <typename T>
void launch_contract(const Seg* segs, const Tile* tiles, int ntiles, const SrcArgs<T>& src,
                     int64_t ns, int splits, cudaStream_t st);
// Register-blocked FP32 projection (mixed path).  Returns false, launching nothing, where it
// does not apply: more than 20 directions in a block, block offsets (offsets_aligned) or the
// row stride not multiples of 4 floats, or sample arrays not 16-byte aligned.
bool launch_project_rb(const float* O, const float* G, int64_t ld, const float* shift32,
                       const ProjBlock* blocks, int nblocks, bool offsets_aligned,
                       const double* cen, float* Y, float* Z, int64_t ldout, int64_t ns,
                       int max_nd, cudaStream_t st);
template <typename T, typename TO>
void launch_project(const T* O, const T* G, int64_t ldo, int64_t ldg, const double* shift,
                    const float* shift32,
                    const ProjBlock* blocks, int nblocks, const double* cen, TO* Y, TO* Z,
                    int64_t ldout, int64_t ns, int max_m, int max_nd, cudaStream_t st);
// Split operands of a chunk (blm_prep.cu): rows of row_bytes per parameter, 128 bytes per
// sample group -- BF16 (tf32 = 0): 32 samples [hi(32) | lo(32)] bf16, a chunk of at most
// row_bytes / 4 samples; TF32 (tf32 = 1): 16 samples [hi(16) | lo(16)] tf32, at most
// row_bytes / 8 samples.  opBS is written only when w is given.  With sY non-null the same pass
// adds the first moments sum w Y', sum w E Y', sum w Z into sY, sEY, sZ (and sum w, sum w E into
// scal if non-null).
void launch_prep(const float* Y, const float* Z, const float* E, const float* w, int64_t ns,
                 int64_t ld, int64_t n, const float* shift32, uint8_t* opA, uint8_t* opBS,
                 uint8_t* opBH, int64_t row_bytes, double* sY, double* sEY, double* sZ,
                 double* scal, int tf32, cudaStream_t st);
// dst[i] = (float)src[i], i < count
void launch_to_f32(const double* src, float* dst, int64_t count, cudaStream_t st);

// ------------------------------- launchers (blm_sweep_tc.cu) ---------------------------------
// One 128 x 256 output tile of a split-precision tcgen05 contraction (blm_sweep_tc.cu):
//   out[r * out_ld + c] += sum_s A(s, r) B(s, c),   r < nA (<= 128), c < nB (<= 256),
// where A is operand rows a_row .. a_row + 127 of prepared operand array a_map and B rows
// b_row .. b_row + 255 of array b_map (prepared rows: one per parameter or direction, see
// launch_prep).  a_view: A's rows lie inside the B rows of the same stage (a_map and b_map hold
// the same data when the sums are unweighted), so A needs no load of its own.
struct TcTile {
  int32_t a_map, b_map;
  int32_t a_row, b_row;
  int32_t nA, nB;
  int32_t a_view;      // 1: A is rows [a_row - b_row, a_row - b_row + 128) of the B stage when
                       //    the launch is unweighted
  int32_t packed;      // 1: a band tile over several blocks (TcPack): out and out_ld unused,
                       //    each product lands in its block's sums if row and column share a
                       //    block (b_map 2: the Hamiltonian half of the block's sums)
  double* out;
  int64_t out_ld;
};
// Block tables of packed tiles: block of each parameter, first parameter, size and sums
// (M_b x 2 M_b) of each block.
struct TcPack {
  const int32_t* blk_of;
  const int64_t* lo;
  const int32_t* m;
  double* const* C;
};
// Operand arrays of one tensor-core launch (up to kTcMaps prepared arrays, rows x row_bytes).
constexpr int kTcMaps = 6;
struct TcOperands {
  const uint8_t* op[kTcMaps];
  int64_t rows[kTcMaps];
};
// Tensor-core contraction of prepared operands (blm_sweep_tc.cu, tc_op_kernel); tf32 selects
// the TF32 split (operands prepared with launch_prep(..., tf32 = 1)).
// wait_limit: polls of a pipeline wait before the kernel gives up and records a timeout in *err
// (BLM_WAIT_LIMIT_DEFAULT normally; 0 gives up at the first wait).
// max_range: longest sample range of a work unit (a multiple of 2048, tuned per problem).
cudaError_t launch_tc_prepared(const TcOperands& ops, int64_t row_bytes, int64_t ns,
                               const TcTile* tiles, int ntiles, int weighted, int32_t* err,
                               uint32_t wait_limit, int tf32, const TcPack& pack,
                               int64_t max_range, cudaStream_t st);

// ------------------------------- launchers (blm_assemble.cu) ---------------------------------
struct BlockAsm {
  int64_t lo;          // first parameter
  int32_t m;           // M_b
  int32_t d;           // tangent dimension M_b + N_O (N_B - 1)
  int32_t b;           // block index
  int32_t pad;
  const double* C;     // M_b x 2 M_b sums  [O'O'^T | O'X'^T]
  double* S;           // (1+d)^2 output
  double* H;           // (1+d)^2 output
};
struct HistSums {      // history sums (N_O > 0), R = N_O * N_B virtual columns t_jk, r = k*N_O+j
  int32_t n_old, n_blocks;
  const double* OT;    // n x 2R: [sum w O' T' | sum w O' (E T' + U)]
  const double* XT;    // n x R : sum w X' T'
  const double* TT;    // R x 2R: [sum w T' T' | sum w T' (E T' + U)]
  const double* sT;    // R: sum w T'
  const double* sET;   // R: sum w E T'
  const double* sU;    // R: sum w U
  const double* gram;  // R x R: D_jk . D_j'k' (zero unless k == k')
};
void launch_assemble_blocks(const BlockAsm* blocks, int nblocks, int max_dim, const double* sO,
                            const double* sEO, const double* sG, const double* scal,
                            HistSums hist, double shift, cudaStream_t st);
void launch_assemble_combined(int64_t dc, const double* C, const double* sY, const double* sEY,
                              const double* sZ, const double* scal, const double* gram,
                              double shift, double* S, double* H, cudaStream_t st);

// ------------------------------- launchers (blm_eig.cu) --------------------------------------
struct EigProblem {
  int32_t m;           // dimension (1 + tangent)
  int32_t k;           // directions wanted (lowest real parts)
  int32_t mode;        // 0: block (complex pair -> Re, Im), 1: combined (lowest must be real)
  int32_t flags;       // kEigLocate32 | kEigUnitS (below)
  const double* S;     // m x m row-major
  const double* H;     // m x m row-major
  double* work;        // 5 m^2 + 16 m doubles
  double* lam;         // k outputs (real parts)
  double* vec;         // k x m outputs (real eigenvectors in the original basis)
  int32_t* status;     // one word
  const int32_t* run_if_noconv;  // if set: solve only when *run_if_noconv == ST_NOCONV (the
                                 // dense fallback after a Davidson run, decided on the device)
};
// EigProblem::flags.  kEigLocate32: an FP32 QR locates the eigenvalues and FP64 inverse
// iteration recomputes the kept ones; the double-word QR runs only when that location cannot be
// trusted (a kept vector that does not converge, or kept eigenvalues closer to each other or to
// the first one left out than the FP32 values can resolve).  kEigUnitS: S is the identity (the
// Davidson projection's S-orthonormal basis), so the Cholesky reduction is skipped.
constexpr int32_t kEigLocate32 = 1;
constexpr int32_t kEigUnitS = 2;
// Launches the dense solver on nprob problems.  With their dimensions (host) and a control
// buffer (device, eig_team_ctl_bytes(nprob)) the largest problems are solved by teams of CTAs
// of one cooperative launch; otherwise one CTA per problem.
void launch_eig(const EigProblem* probs, int nprob, int threads, cudaStream_t st,
                const int32_t* dims = nullptr, void* team_ctl = nullptr);
size_t eig_team_ctl_bytes(int nprob);
size_t eig_work_doubles(int64_t m);
// Lowest eigenpair by generalized Davidson (k = 1, mode 1) of the one problem *probs, whose
// workspace `work` (device, davidson_work_doubles(m) doubles) and dimension m the caller passes
// (no read-back: the launch is stream-ordered and can be captured in a graph).
cudaError_t launch_davidson(const EigProblem* probs, double tol, int max_iter, double* work, int m,
                            cudaStream_t st);
size_t davidson_work_doubles(int64_t m);

// ------------------------------- launchers (blm_update.cu) -----------------------------------
struct DirBlock {       // block solve -> B rows
  int32_t m;            // M_b
  int32_t k;            // kept
  int32_t d1;           // 1 + d_b (eigenvector length)
  int32_t pad;
  const double* vec;    // k x d1 eigenvectors
  double* B;            // k x M_b output rows
  int32_t* status;
};
void launch_extract_dirs(const DirBlock* blocks, int nblocks, cudaStream_t st);
void launch_cen(const ProjBlock* blocks, int nblocks, const double* sO, const double* scal,
                double* cen, cudaStream_t st);
void launch_gram(const ProjBlock* blocks, int nblocks, int max_nd, double* gram, int64_t ld,
                 cudaStream_t st);
void launch_update(int nblocks, const ProjBlock* blocks, int64_t dc, const double* c,
                   const double* shift, const double* sO, const double* scal, double* alpha,
                   double* dmu, int32_t* status, cudaStream_t st);

}  // namespace blm
