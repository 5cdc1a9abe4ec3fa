// C ABI of the blocked-linear-method library (declared in include/blm.h).
//
// The handle owns every device buffer of one optimisation step; the calls only enqueue kernels
// on the handle's stream (the solves also synchronise to report numeric status).  Sample chunks
// handed in as host memory are staged through two device buffers on a copy stream.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <type_traits>
#include <vector>

#include "blm_internal.cuh"

using namespace blm;

namespace {

enum State { ST_CREATED = 0, ST_ACCUM = 1, ST_BLOCKS = 2, ST_PROJ = 3, ST_DONE = 4 };

constexpr int64_t kSubChunk = 65536;     // samples per scratch pass (history / projection)
constexpr int64_t kShiftSamples = 65536; // samples that fix the reference shift
// Combined problems up to this dimension use the dense solver (exact ordering of the whole
// spectrum); larger ones use generalized Davidson for the lowest eigenpair.
constexpr int64_t kDenseCombinedMax = 320;
constexpr double kDavidsonTol = 1e-11;
constexpr int kDavidsonIter = 400;

struct Alloc {
  // sizes in bytes of every device buffer; filled by plan()
  size_t total = 0;
  std::vector<std::pair<void**, size_t>> items;
  void add(void** p, size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    items.emplace_back(p, bytes);
    total += bytes;
  }
};

}  // namespace

struct blm_handle {
  // problem
  int64_t n = 0;
  int nb = 0;
  std::vector<int64_t> off;
  int K = 0;
  int n_old = 0;
  int prec = 0;
  int in_type = 0;
  double shift = 0.0;
  cudaStream_t st = nullptr;
  int device = 0;
  int state = ST_CREATED;
  bool shift_set = false;
  std::string err;
  // derived sizes
  std::vector<int> Mb, Kb, db, oc;
  std::vector<int64_t> C_off, SH_off, eigw_off, vec_off, B_off, lam_off;
  int64_t dc = 0;      // combined tangent dimension
  int R = 0;           // history virtual columns N_O * N_B
  int maxM = 0, maxD = 0, maxK = 0;
  size_t elem = 8;     // input element size
  size_t selem = 8;    // scratch element size (8 FP64 path, 4 mixed path)
  // device buffers
  double* d_shift = nullptr;
  float* d_shift32 = nullptr;
  float* d_B32 = nullptr;                   // B^(b) rows in FP32 (mixed-path projection)
  uint8_t* d_opA = nullptr;                 // prepared split-BF16 operands of a sub-chunk
  uint8_t* d_opBS = nullptr;                //   (BF16X4 first sweep): Y', w Y', w X' rows
  uint8_t* d_opBH = nullptr;
  int64_t op_row_bytes = 0;                 //   bytes per parameter row (kSubChunk / 32 x 128)
  int64_t B_words = 0;                      // doubles in d_B
  double* d_colsum = nullptr;
  double* d_vec = nullptr;       // sO | sEO | sG  (3n)
  double* d_scal = nullptr;      // [sw, sE, count, alpha]
  double* d_C = nullptr;         // block sums
  double* d_D = nullptr;         // history directions n_old x n
  double* d_OT = nullptr;        // n x 2R
  double* d_XT = nullptr;        // n x R
  double* d_TT = nullptr;        // R x 2R
  double* d_hvec = nullptr;      // sT | sET | sU (3R)
  double* d_hgram = nullptr;     // R x R
  void* d_scrY = nullptr;        // kSubChunk x max(R, dc)
  void* d_scrZ = nullptr;
  double* d_S = nullptr;         // block S matrices
  double* d_H = nullptr;
  double* d_eigw = nullptr;
  double* d_lam = nullptr;
  double* d_evec = nullptr;
  double* d_B = nullptr;
  int32_t* d_status = nullptr;   // nb + 4 words
  double* d_Cc = nullptr;        // dc x 2dc
  double* d_cvec = nullptr;      // sY | sEY | sZ (3 dc)
  double* d_cen = nullptr;       // dc
  double* d_cgram = nullptr;     // dc x dc
  double* d_Sc = nullptr;
  double* d_Hc = nullptr;
  double* d_ceigw = nullptr;
  double* d_clam = nullptr;
  double* d_cev = nullptr;
  double* d_dmu = nullptr;
  // device tables
  Seg* d_seg1 = nullptr;  int nseg1 = 0;    // pass-1 block segments
  Tile* d_tile1 = nullptr; int ntile1 = 0;
  Seg* d_segh = nullptr;  int nsegh = 0;    // history segments
  Tile* d_tileh = nullptr; int ntileh = 0;
  Seg* d_segc = nullptr;  int nsegc = 0;    // combined segments
  Tile* d_tilec = nullptr; int ntilec = 0;
  ProjBlock* d_pbB = nullptr;               // B^(b) directions
  ProjBlock* d_pbD = nullptr;               // history directions
  BlockAsm* d_asm = nullptr;
  EigProblem* d_eigp = nullptr;
  EigProblem* d_ceigp = nullptr;
  DirBlock* d_dirb = nullptr;
  TcTile* d_tc1 = nullptr;  int ntc1 = 0;   // pass-1 tensor-core tiles
  TcTile* d_tc2 = nullptr;  int ntc2 = 0;   // combined tensor-core tiles
  int off_aligned = 0;                     // block offsets all multiples of 4
  // host staging
  void* d_stage[2][4] = {{nullptr}};
  int64_t stage_rows = 0;
  cudaStream_t copy_st = nullptr;
  cudaEvent_t ev_copy[2] = {nullptr, nullptr};
  cudaEvent_t ev_done[2] = {nullptr, nullptr};
  void* base = nullptr;   // single device allocation
  // profiling
  bool prof = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_ev;
  std::vector<cudaEvent_t> ev_pool;
  int64_t prof_launch[BLM_PROF_CLASSES] = {0};
};

namespace {

enum ProfClass {
  PC_SHIFT = 0, PC_SUMS = 1, PC_CONTRACT = 2, PC_TC1 = 3, PC_HIST = 4, PC_ASSEMBLE = 5,
  PC_EIG_BLOCKS = 6, PC_DIRS = 7, PC_PROJECT = 8, PC_TC2 = 9, PC_EIG_COMBINED = 10, PC_UPDATE = 11,
  PC_PREP = 12
};
const char* kProfNames[BLM_PROF_CLASSES] = {
    "reference_shift", "first_moments", "contract_f64", "contract_tc_pass1", "history_terms",
    "assemble", "eig_blocks", "directions", "project", "contract_tc_pass2", "eig_combined",
    "update", "operand_prep"};

cudaEvent_t pool_event(blm_handle* h) {
  if (!h->ev_pool.empty()) {
    cudaEvent_t e = h->ev_pool.back();
    h->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

// Brackets the launches of one kernel class with events when profiling is on.
struct Prof {
  blm_handle* h;
  int cls;
  int n;
  cudaEvent_t a = nullptr, b = nullptr;
  Prof(blm_handle* hh, int c, int launches = 1) : h(hh), cls(c), n(launches) {
    if (h->prof) {
      a = pool_event(h);
      b = pool_event(h);
      cudaEventRecord(a, h->st);
    }
  }
  ~Prof() {
    if (h->prof) {
      cudaEventRecord(b, h->st);
      h->prof_ev.push_back({cls, {a, b}});
      h->prof_launch[cls] += n;
    }
  }
};

blm_status fail(blm_handle* h, blm_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}

blm_status cuda_fail(blm_handle* h, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  if (h) h->err = m;
  return BLM_ERR_CUDA;
}

#define BLM_CU(h, call)                                    \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
  } while (0)

blm_status validate(const blm_problem* p, std::string& why) {
  if (!p) { why = "problem is NULL"; return BLM_ERR_ARG; }
  if (p->n_params <= 0) { why = "n_params must be positive"; return BLM_ERR_ARG; }
  if (p->n_blocks <= 0 || p->n_blocks > p->n_params) { why = "bad n_blocks"; return BLM_ERR_ARG; }
  if (!p->block_offsets) { why = "block_offsets is NULL"; return BLM_ERR_ARG; }
  if (p->block_offsets[0] != 0 || p->block_offsets[p->n_blocks] != p->n_params) {
    why = "block_offsets must start at 0 and end at n_params";
    return BLM_ERR_ARG;
  }
  for (int b = 0; b < p->n_blocks; ++b)
    if (p->block_offsets[b + 1] <= p->block_offsets[b]) {
      why = "block_offsets must increase";
      return BLM_ERR_ARG;
    }
  if (p->n_keep <= 0 || p->n_keep > 64) { why = "n_keep must be in 1..64"; return BLM_ERR_ARG; }
  if (p->n_old < 0 || p->n_old > 16) { why = "n_old must be in 0..16"; return BLM_ERR_ARG; }
  if (p->n_old > 0 && !p->old_dirs) { why = "old_dirs is NULL"; return BLM_ERR_ARG; }
  if (p->n_old > 0 && p->n_blocks < 2) { why = "history directions need >= 2 blocks"; return BLM_ERR_ARG; }
  if (p->precision != BLM_PREC_F64 && p->precision != BLM_PREC_BF16X4 &&
      p->precision != BLM_PREC_TF32X3) {
    why = "unknown precision";
    return BLM_ERR_ARG;
  }
  if (p->input_type != BLM_IN_F64 && p->input_type != BLM_IN_F32) {
    why = "unknown input_type";
    return BLM_ERR_ARG;
  }
  if (p->precision != BLM_PREC_F64 && p->input_type != BLM_IN_F32) {
    why = "the split-precision tensor-core paths take FP32 inputs";
    return BLM_ERR_UNSUPPORTED;
  }
  if (p->precision != BLM_PREC_F64 && p->n_old > 0) {
    why = "history directions run on the FP64 path only";
    return BLM_ERR_UNSUPPORTED;
  }
  if (!(p->shift >= 0.0) || !isfinite(p->shift)) { why = "shift must be finite and >= 0"; return BLM_ERR_ARG; }
  for (int b = 0; b < p->n_blocks; ++b) {
    const int64_t m = p->block_offsets[b + 1] - p->block_offsets[b];
    const int64_t d = m + (int64_t)p->n_old * (p->n_blocks - 1);
    if (d + 1 > 4096) { why = "a block problem exceeds dimension 4096"; return BLM_ERR_UNSUPPORTED; }
  }
  return BLM_OK;
}

void derive(blm_handle* h, const blm_problem* p) {
  h->n = p->n_params;
  h->nb = p->n_blocks;
  h->off.assign(p->block_offsets, p->block_offsets + p->n_blocks + 1);
  h->off_aligned = 1;
  for (int64_t o : h->off)
    if (o % 4 != 0) h->off_aligned = 0;
  h->K = p->n_keep;
  h->n_old = p->n_old;
  h->prec = p->precision;
  h->in_type = p->input_type;
  h->shift = p->shift;
  h->elem = p->input_type == BLM_IN_F32 ? 4 : 8;
  h->selem = p->precision == BLM_PREC_F64 ? 8 : 4;
  h->R = p->n_old * p->n_blocks;
  h->Mb.resize(h->nb);
  h->Kb.resize(h->nb);
  h->db.resize(h->nb);
  h->oc.resize(h->nb);
  h->C_off.resize(h->nb);
  h->SH_off.resize(h->nb);
  h->eigw_off.resize(h->nb);
  h->vec_off.resize(h->nb);
  h->B_off.resize(h->nb);
  h->lam_off.resize(h->nb);
  int64_t c = 0, sh = 0, ew = 0, vo = 0, bo = 0, lo = 0, occ = 0;
  h->maxM = h->maxD = h->maxK = 0;
  for (int b = 0; b < h->nb; ++b) {
    const int m = (int)(h->off[b + 1] - h->off[b]);
    h->Mb[b] = m;
    h->Kb[b] = std::min(h->K, m);
    h->db[b] = m + h->n_old * (h->nb - 1);
    h->oc[b] = (int)occ;
    occ += h->Kb[b];
    const int64_t D = h->db[b] + 1;
    h->C_off[b] = c;        c += 2LL * m * m;
    h->SH_off[b] = sh;      sh += D * D;
    h->eigw_off[b] = ew;    ew += (int64_t)eig_work_doubles(D);
    h->vec_off[b] = vo;     vo += (int64_t)h->Kb[b] * D;
    h->B_off[b] = bo;       bo += (int64_t)h->Kb[b] * m;
    h->lam_off[b] = lo;     lo += h->Kb[b];
    h->maxM = std::max(h->maxM, m);
    h->maxD = std::max(h->maxD, h->db[b]);
    h->maxK = std::max(h->maxK, h->Kb[b]);
  }
  h->dc = occ;
}

// Pass-1 contraction tiles of the FP64 path: per block, 64 x 64 tiles of [O'O'^T | O'X'^T].
void build_pass1_tables(blm_handle* h, std::vector<Seg>& segs, std::vector<Tile>& tiles,
                        double* C_base) {
  for (int b = 0; b < h->nb; ++b) {
    const int m = h->Mb[b];
    const int i_so = (int)segs.size();
    segs.push_back(Seg{0, 0, h->off[b]});
    segs.push_back(Seg{0, 1, h->off[b]});
    double* Cb = C_base + h->C_off[b];
    for (int i0 = 0; i0 < m; i0 += 64)
      for (int half = 0; half < 2; ++half)
        for (int j0 = 0; j0 < m; j0 += 64) {
          Tile t{};
          t.a_seg = i_so;
          t.b_seg = i_so + half;
          t.a0 = i0;
          t.b0 = j0;
          t.a_n = std::min(64, m - i0);
          t.b_n = std::min(64, m - j0);
          t.out = Cb + (int64_t)i0 * 2 * m + half * m + j0;
          t.out_ld = 2 * m;
          tiles.push_back(t);
        }
  }
}

// Generic tiles for out = sum w A(s, i) B(s, j) with A one segment of `rows` columns and B a
// list of segments of `cols` columns each, laid side by side in out.
void add_tiles(std::vector<Tile>& tiles, int a_seg, int rows, const std::vector<int>& b_segs,
               int cols, double* out, int64_t ld) {
  for (int i0 = 0; i0 < rows; i0 += 64)
    for (size_t q = 0; q < b_segs.size(); ++q)
      for (int j0 = 0; j0 < cols; j0 += 64) {
        Tile t{};
        t.a_seg = a_seg;
        t.b_seg = b_segs[q];
        t.a0 = i0;
        t.b0 = j0;
        t.a_n = std::min(64, rows - i0);
        t.b_n = std::min(64, cols - j0);
        t.out = out + (int64_t)i0 * ld + (int64_t)q * cols + j0;
        t.out_ld = ld;
        tiles.push_back(t);
      }
}

template <typename V>
blm_status upload(blm_handle* h, const std::vector<V>& v, V** dst) {
  if (v.empty()) return BLM_OK;
  BLM_CU(h, cudaMalloc((void**)dst, sizeof(V) * v.size()));
  BLM_CU(h, cudaMemcpy(*dst, v.data(), sizeof(V) * v.size(), cudaMemcpyHostToDevice));
  return BLM_OK;
}

void plan(blm_handle* h, Alloc& a) {
  const int64_t n = h->n;
  const int64_t Csz = h->C_off.empty() ? 0 : h->C_off.back() + 2LL * h->Mb.back() * h->Mb.back();
  const int64_t SHsz = h->SH_off.back() + (int64_t)(h->db.back() + 1) * (h->db.back() + 1);
  const int64_t EWsz = h->eigw_off.back() + (int64_t)eig_work_doubles(h->db.back() + 1);
  const int64_t VOsz = h->vec_off.back() + (int64_t)h->Kb.back() * (h->db.back() + 1);
  const int64_t BOsz = h->B_off.back() + (int64_t)h->Kb.back() * h->Mb.back();
  h->B_words = BOsz;
  const int64_t LOsz = h->lam_off.back() + h->Kb.back();
  const int64_t dc = h->dc, R = h->R;
  const int64_t scr_cols = std::max<int64_t>(dc, R);
  a.add((void**)&h->d_shift, 8 * n);
  a.add((void**)&h->d_shift32, 4 * n);
  a.add((void**)&h->d_colsum, 8 * n);
  a.add((void**)&h->d_vec, 8 * 3 * n);
  a.add((void**)&h->d_scal, 8 * 8);
  a.add((void**)&h->d_C, 8 * Csz);
  if (h->n_old > 0) {
    a.add((void**)&h->d_D, 8 * h->n_old * n);
    a.add((void**)&h->d_OT, 8 * n * 2 * R);
    a.add((void**)&h->d_XT, 8 * n * R);
    a.add((void**)&h->d_TT, 8 * R * 2 * R);
    a.add((void**)&h->d_hvec, 8 * 3 * R);
    a.add((void**)&h->d_hgram, 8 * R * R);
  }
  a.add((void**)&h->d_scrY, h->selem * kSubChunk * scr_cols);
  a.add((void**)&h->d_scrZ, h->selem * kSubChunk * scr_cols);
  a.add((void**)&h->d_S, 8 * SHsz);
  a.add((void**)&h->d_H, 8 * SHsz);
  a.add((void**)&h->d_eigw, 8 * EWsz);
  a.add((void**)&h->d_lam, 8 * LOsz);
  a.add((void**)&h->d_evec, 8 * VOsz);
  a.add((void**)&h->d_B, 8 * BOsz);
  a.add((void**)&h->d_B32, 4 * BOsz);
  if (h->prec == BLM_PREC_BF16X4 && h->in_type == BLM_IN_F32) {
    h->op_row_bytes = kSubChunk / 32 * 128;
    a.add((void**)&h->d_opA, h->op_row_bytes * n);
    a.add((void**)&h->d_opBS, h->op_row_bytes * n);
    a.add((void**)&h->d_opBH, h->op_row_bytes * n);
  }
  a.add((void**)&h->d_status, 4 * (h->nb + 8));
  a.add((void**)&h->d_Cc, 8 * dc * 2 * dc);
  a.add((void**)&h->d_cvec, 8 * 3 * dc);
  a.add((void**)&h->d_cen, 8 * dc);
  a.add((void**)&h->d_cgram, 8 * dc * dc);
  a.add((void**)&h->d_Sc, 8 * (dc + 1) * (dc + 1));
  a.add((void**)&h->d_Hc, 8 * (dc + 1) * (dc + 1));
  a.add((void**)&h->d_ceigw, 8 * std::max(eig_work_doubles(dc + 1), davidson_work_doubles(dc + 1)));
  a.add((void**)&h->d_clam, 8 * 4);
  a.add((void**)&h->d_cev, 8 * (dc + 1));
  a.add((void**)&h->d_dmu, 8 * n);
}

blm_status zero_sums(blm_handle* h) {
  const int64_t Csz = h->C_off.back() + 2LL * h->Mb.back() * h->Mb.back();
  BLM_CU(h, cudaMemsetAsync(h->d_vec, 0, 8 * 3 * h->n, h->st));
  BLM_CU(h, cudaMemsetAsync(h->d_scal, 0, 8 * 8, h->st));
  BLM_CU(h, cudaMemsetAsync(h->d_C, 0, 8 * Csz, h->st));
  BLM_CU(h, cudaMemsetAsync(h->d_colsum, 0, 8 * h->n, h->st));
  if (h->n_old > 0) {
    const int64_t n = h->n, R = h->R;
    BLM_CU(h, cudaMemsetAsync(h->d_OT, 0, 8 * n * 2 * R, h->st));
    BLM_CU(h, cudaMemsetAsync(h->d_XT, 0, 8 * n * R, h->st));
    BLM_CU(h, cudaMemsetAsync(h->d_TT, 0, 8 * R * 2 * R, h->st));
    BLM_CU(h, cudaMemsetAsync(h->d_hvec, 0, 8 * 3 * R, h->st));
  }
  BLM_CU(h, cudaMemsetAsync(h->d_Cc, 0, 8 * h->dc * 2 * h->dc, h->st));
  BLM_CU(h, cudaMemsetAsync(h->d_cvec, 0, 8 * 3 * h->dc, h->st));
  BLM_CU(h, cudaMemsetAsync(h->d_status, 0, 4 * (h->nb + 8), h->st));
  h->shift_set = false;
  h->state = ST_CREATED;
  return BLM_OK;
}

__global__ void finalize_shift_kernel(const double* colsum, int64_t n, double count, int f32,
                                      double* shift, float* shift32) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double c = colsum[i] / count;
  if (f32) c = (double)(float)c;
  shift[i] = c;
  shift32[i] = (float)c;
}

int pick_splits(int ntiles, int64_t ns, int64_t min_per) {
  const int64_t target = 4 * 152;
  int64_t s = (target + ntiles - 1) / std::max(ntiles, 1);
  s = std::min<int64_t>(s, std::max<int64_t>(1, ns / min_per));
  return (int)std::max<int64_t>(1, s);
}

// ---------------------------------------------------------------------------------------------
// Device-pointer sweeps.
// ---------------------------------------------------------------------------------------------
template <typename T>
blm_status accumulate_dev(blm_handle* h, const T* O, const T* G, const T* E, const T* w,
                          int64_t ns, int64_t ld) {
  cudaStream_t st = h->st;
  if (!h->shift_set) {
    const int64_t cnt = std::min(ns, kShiftSamples);
    Prof pr(h, PC_SHIFT, 2);
    launch_colmean<T>(O, cnt, ld, h->n, h->d_colsum, st);
    finalize_shift_kernel<<<(unsigned)((h->n + 255) / 256), 256, 0, st>>>(
        h->d_colsum, h->n, (double)cnt, h->in_type == BLM_IN_F32, h->d_shift, h->d_shift32);
    h->shift_set = true;
  }
  const bool mixed = h->prec != BLM_PREC_F64;
  const bool prepared = mixed && h->d_opA != nullptr;   // first moments fused into the prep pass
  if (!prepared) {
    Prof pr(h, PC_SUMS);
    launch_sums<T>(O, G, E, w, ns, ld, ld, h->n, h->d_shift, h->d_vec, h->d_vec + h->n,
                   h->d_vec + 2 * h->n, h->d_scal, mixed, st);
  }
  if (h->prec == BLM_PREC_F64) {
    // FP64 path (FP64 inputs, or FP32 inputs widened on load): block contractions and history
    // terms on CUDA cores
    SrcArgs<T> src{O, nullptr, G, nullptr, {ld, 0}, h->d_shift, E, w};
    {
      Prof pr(h, PC_CONTRACT);
      launch_contract(h->d_seg1, h->d_tile1, h->ntile1, src, ns, pick_splits(h->ntile1, ns, 512),
                      st);
    }
    if (h->n_old > 0) {
      const int64_t R = h->R;
      double* TY = (double*)h->d_scrY;
      double* TZ = (double*)h->d_scrZ;
      for (int64_t s0 = 0; s0 < ns; s0 += kSubChunk) {
        const int64_t cnt = std::min(kSubChunk, ns - s0);
        const T* Os = O + s0 * ld;
        const T* Gs = G + s0 * ld;
        const T* Es = E + s0;
        const T* ws = w ? w + s0 : nullptr;
        // t_jk = O'_k . D_jk and u_jk = G_k . D_jk (Eq. 9 ratios) for every block k
        Prof pr(h, PC_HIST, 3);
        launch_project<T, double>(Os, Gs, ld, ld, h->d_shift, nullptr, h->d_pbD, h->nb, nullptr, TY,
                                  TZ, R, cnt, h->maxM, h->n_old, st);
        launch_sums_mixed<T>(TY, TZ, Es, ws, cnt, R, h->d_hvec, h->d_hvec + R, h->d_hvec + 2 * R,
                             st);
        SrcArgs<T> hs{Os, TY, Gs, TZ, {ld, R}, h->d_shift, Es, ws};
        launch_contract(h->d_segh, h->d_tileh, h->ntileh, hs, cnt,
                        pick_splits(h->ntileh, cnt, 512), st);
      }
    }
  } else if (h->d_opA) {
    // split-BF16: operands prepared once per element, then TMA + tensor cores
    for (int64_t s0 = 0; s0 < ns; s0 += kSubChunk) {
      const int64_t cnt = std::min(kSubChunk, ns - s0);
      const float* Wp = w ? (const float*)w + s0 : nullptr;
      {
        Prof pr(h, PC_PREP);
        launch_prep((const float*)O + s0 * ld, (const float*)G + s0 * ld, (const float*)E + s0, Wp,
                    cnt, ld, h->n, h->d_shift32, h->d_opA, h->d_opBS, h->d_opBH, h->op_row_bytes,
                    h->d_vec, h->d_vec + h->n, h->d_vec + 2 * h->n, h->d_scal, st);
      }
      Prof pr(h, PC_TC1);
      cudaError_t e = launch_tc_prepared(h->d_opA, h->d_opBS, h->d_opBH, h->n, h->op_row_bytes,
                                         cnt, h->d_tc1, h->ntc1, Wp != nullptr,
                                         h->d_status + h->nb + 2, st);
      if (e != cudaSuccess) return cuda_fail(h, e, "launch_tc_prepared");
    }
  } else {
    if (!tc_supported()) return fail(h, BLM_ERR_UNSUPPORTED, "tensor-core path not built");
    Prof pr(h, PC_TC1);
    cudaError_t e = launch_tc_accumulate((const float*)O, (const float*)G, (const float*)E,
                                         (const float*)w, ns, h->n, ld, h->d_shift32, h->d_tc1,
                                         h->ntc1, h->d_status + h->nb + 2,
                                         h->prec == BLM_PREC_TF32X3, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "launch_tc_accumulate");
  }
  return BLM_OK;
}

template <typename T>
blm_status project_dev(blm_handle* h, const T* O, const T* G, const T* E, const T* w,
                       int64_t ns, int64_t ld) {
  cudaStream_t st = h->st;
  const int64_t dc = h->dc;
  for (int64_t s0 = 0; s0 < ns; s0 += kSubChunk) {
    const int64_t cnt = std::min(kSubChunk, ns - s0);
    const T* Os = O + s0 * ld;
    const T* Gs = G + s0 * ld;
    const T* Es = E + s0;
    const T* ws = w ? w + s0 : nullptr;
    if (h->prec == BLM_PREC_F64) {
      // p_bj = Obar_b . B_j (centred with the first sweep's mean) and r_bj = G_b . B_j (Eq. 6)
      double* PY = (double*)h->d_scrY;
      double* PZ = (double*)h->d_scrZ;
      {
        Prof pr(h, PC_PROJECT, 2);
        launch_project<T, double>(Os, Gs, ld, ld, h->d_shift, nullptr, h->d_pbB, h->nb, h->d_cen, PY,
                                  PZ, dc, cnt, h->maxM, h->maxK, st);
        launch_sums_mixed<T>(PY, PZ, Es, ws, cnt, dc, h->d_cvec, h->d_cvec + dc,
                             h->d_cvec + 2 * dc, st);
      }
      SrcArgs<T> cs{nullptr, PY, nullptr, PZ, {0, dc}, nullptr, Es, ws};
      Prof pr(h, PC_CONTRACT);
      launch_contract(h->d_segc, h->d_tilec, h->ntilec, cs, cnt,
                      pick_splits(h->ntilec, cnt, 512), st);
    } else if constexpr (std::is_same<T, float>::value) {
      // mixed paths (FP32 inputs only)
      float* PY = (float*)h->d_scrY;
      float* PZ = (float*)h->d_scrZ;
      const bool prepared = h->d_opA && dc <= h->n;
      {
        Prof pr(h, PC_PROJECT, prepared ? 1 : 2);
        if (!launch_project_rb(Os, Gs, ld, h->d_shift ? h->d_shift32 : nullptr, h->d_pbB, h->nb,
                               h->off_aligned != 0, h->d_cen, PY, PZ, dc, cnt, h->maxK, st))
          launch_project<float, float>(Os, Gs, ld, ld, h->d_shift, h->d_shift32, h->d_pbB, h->nb,
                                       h->d_cen, PY, PZ, dc, cnt, h->maxM, h->maxK, st);
        if (!prepared)
          launch_sums<float>(PY, PZ, Es, ws, cnt, dc, dc, dc, nullptr, h->d_cvec, h->d_cvec + dc,
                             h->d_cvec + 2 * dc, nullptr, true, st);
      }
      if (prepared) {
        // split-BF16: the projections p (already centred) and r take the first sweep's route,
        // prepared operands (no shift) then TMA + tensor cores
        {
          Prof pr(h, PC_PREP);
          launch_prep(PY, PZ, Es, ws, cnt, dc, dc, nullptr, h->d_opA, h->d_opBS, h->d_opBH,
                      h->op_row_bytes, h->d_cvec, h->d_cvec + dc, h->d_cvec + 2 * dc, nullptr, st);
        }
        Prof pr(h, PC_TC2);
        cudaError_t e = launch_tc_prepared(h->d_opA, h->d_opBS, h->d_opBH, dc, h->op_row_bytes,
                                           cnt, h->d_tc2, h->ntc2, ws != nullptr,
                                           h->d_status + h->nb + 2, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "launch_tc_prepared (combined)");
      } else {
        Prof pr(h, PC_TC2);
        cudaError_t e = launch_tc_accumulate(PY, PZ, Es, ws, cnt, dc, dc, nullptr, h->d_tc2,
                                             h->ntc2, h->d_status + h->nb + 2,
                                             h->prec == BLM_PREC_TF32X3, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "launch_tc_accumulate (combined)");
      }
    }
  }
  return BLM_OK;
}

bool is_device_ptr(const void* p) {
  if (!p) return true;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T>
blm_status sweep(blm_handle* h, int pass, const void* O, const void* G, const void* E,
                 const void* w, int64_t ns, int64_t ld) {
  if (ns == 0) return BLM_OK;
  const bool dev = is_device_ptr(O);
  if (dev != is_device_ptr(G) || dev != is_device_ptr(E) || (w && dev != is_device_ptr(w)))
    return fail(h, BLM_ERR_ARG, "sample arrays must all be device or all be host memory");
  if (dev) {
    if (pass == 1) return accumulate_dev<T>(h, (const T*)O, (const T*)G, (const T*)E, (const T*)w, ns, ld);
    return project_dev<T>(h, (const T*)O, (const T*)G, (const T*)E, (const T*)w, ns, ld);
  }
  // host memory: stage through two device buffers
  const size_t es = sizeof(T);
  if (!h->d_stage[0][0]) {
    // pieces of 256 MiB: the copies run at the host link's rate (about 210 GB/s measured) at
    // this size already, and larger pieces measured no faster end to end
    const int64_t row = (int64_t)(2 * h->n + 2) * es;
    int64_t rows = std::max<int64_t>(256, ((int64_t)256 << 20) / row);
    rows = std::min<int64_t>(rows, kSubChunk);
    h->stage_rows = rows;
    for (int b = 0; b < 2; ++b) {
      BLM_CU(h, cudaMalloc(&h->d_stage[b][0], es * rows * h->n));
      BLM_CU(h, cudaMalloc(&h->d_stage[b][1], es * rows * h->n));
      BLM_CU(h, cudaMalloc(&h->d_stage[b][2], es * rows));
      BLM_CU(h, cudaMalloc(&h->d_stage[b][3], es * rows));
      BLM_CU(h, cudaEventCreateWithFlags(&h->ev_copy[b], cudaEventDisableTiming));
      BLM_CU(h, cudaEventCreateWithFlags(&h->ev_done[b], cudaEventDisableTiming));
    }
    BLM_CU(h, cudaStreamCreateWithFlags(&h->copy_st, cudaStreamNonBlocking));
    BLM_CU(h, cudaEventRecord(h->ev_done[0], h->st));
    BLM_CU(h, cudaEventRecord(h->ev_done[1], h->st));
  }
  const int64_t rows = h->stage_rows;
  int buf = 0;
  for (int64_t s0 = 0; s0 < ns; s0 += rows, buf ^= 1) {
    const int64_t cnt = std::min(rows, ns - s0);
    BLM_CU(h, cudaStreamWaitEvent(h->copy_st, h->ev_done[buf], 0));
    if (ld == h->n) {   // contiguous rows: one linear copy per array
      BLM_CU(h, cudaMemcpyAsync(h->d_stage[buf][0], (const char*)O + s0 * ld * es,
                                es * h->n * cnt, cudaMemcpyHostToDevice, h->copy_st));
      BLM_CU(h, cudaMemcpyAsync(h->d_stage[buf][1], (const char*)G + s0 * ld * es,
                                es * h->n * cnt, cudaMemcpyHostToDevice, h->copy_st));
    } else {
      BLM_CU(h, cudaMemcpy2DAsync(h->d_stage[buf][0], es * h->n, (const char*)O + s0 * ld * es,
                                  es * ld, es * h->n, cnt, cudaMemcpyHostToDevice, h->copy_st));
      BLM_CU(h, cudaMemcpy2DAsync(h->d_stage[buf][1], es * h->n, (const char*)G + s0 * ld * es,
                                  es * ld, es * h->n, cnt, cudaMemcpyHostToDevice, h->copy_st));
    }
    BLM_CU(h, cudaMemcpyAsync(h->d_stage[buf][2], (const char*)E + s0 * es, es * cnt,
                              cudaMemcpyHostToDevice, h->copy_st));
    if (w)
      BLM_CU(h, cudaMemcpyAsync(h->d_stage[buf][3], (const char*)w + s0 * es, es * cnt,
                                cudaMemcpyHostToDevice, h->copy_st));
    BLM_CU(h, cudaEventRecord(h->ev_copy[buf], h->copy_st));
    BLM_CU(h, cudaStreamWaitEvent(h->st, h->ev_copy[buf], 0));
    const T* dO = (const T*)h->d_stage[buf][0];
    const T* dG = (const T*)h->d_stage[buf][1];
    const T* dE = (const T*)h->d_stage[buf][2];
    const T* dw = w ? (const T*)h->d_stage[buf][3] : nullptr;
    blm_status s = pass == 1 ? accumulate_dev<T>(h, dO, dG, dE, dw, cnt, h->n)
                             : project_dev<T>(h, dO, dG, dE, dw, cnt, h->n);
    if (s != BLM_OK) return s;
    BLM_CU(h, cudaEventRecord(h->ev_done[buf], h->st));
  }
  return BLM_OK;
}

const char* status_text(int s) {
  switch (s) {
    case ST_NOT_PD: return "overlap matrix is not positive definite";
    case ST_NONFINITE: return "non-finite matrix element";
    case ST_COMPLEX: return "lowest eigenvalue is complex";
    case ST_NOCONV: return "QR iteration did not converge";
    case ST_ALPHA: return "alpha ~ 0: update orthogonal to Psi";
    case ST_ZERO_DIR: return "zero update direction";
    default: return "unknown numeric failure";
  }
}

}  // namespace

extern "C" {

size_t blm_memory_estimate(const blm_problem* p) {
  std::string why;
  if (validate(p, why) != BLM_OK) return 0;
  blm_handle h;
  derive(&h, p);
  Alloc a;
  plan(&h, a);
  return a.total;
}

double blm_lm_matrix_bytes(int64_t n_params) {
  const double d = 1.0 + (double)n_params;
  return 2.0 * 8.0 * d * d;
}

double blm_matrix_bytes_dominant(int64_t n_params, int32_t n_blocks, int32_t n_old) {
  const double nv = (double)n_params, nb = (double)n_blocks, no = (double)n_old;
  const double hh = nv * nv / nb + 2.0 * nv * no * (nb - 1.0);
  const double ss = nv * nv / nb + nv * no * (nb - 1.0);
  return 8.0 * (hh + ss);
}

blm_status blm_create(const blm_problem* p, void* stream, blm_handle** out) {
  if (!out) return BLM_ERR_ARG;
  *out = nullptr;
  std::string why;
  blm_status vs = validate(p, why);
  if (vs != BLM_OK) {
    fprintf(stderr, "blm_create: %s\n", why.c_str());
    return vs;
  }
  blm_handle* h = new blm_handle();
  h->st = (cudaStream_t)stream;
  cudaGetDevice(&h->device);
  derive(h, p);
  Alloc a;
  plan(h, a);
  cudaError_t e = cudaMalloc(&h->base, a.total);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return BLM_ERR_NOMEM;
  }
  char* cur = (char*)h->base;
  for (auto& it : a.items) {
    *it.first = cur;
    cur += it.second;
  }
  blm_status s = BLM_OK;
  // history directions
  if (h->n_old > 0) {
    const bool dev = is_device_ptr(p->old_dirs);
    e = cudaMemcpy(h->d_D, p->old_dirs, 8 * h->n_old * h->n,
                   dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
    if (e != cudaSuccess) s = cuda_fail(h, e, "copy old_dirs");
  }
  // tables
  std::vector<Seg> segs;
  std::vector<Tile> tiles;
  build_pass1_tables(h, segs, tiles, h->d_C);
  h->nseg1 = (int)segs.size();
  h->ntile1 = (int)tiles.size();
  if (s == BLM_OK) s = upload(h, segs, &h->d_seg1);
  if (s == BLM_OK) s = upload(h, tiles, &h->d_tile1);
  if (h->n_old > 0) {
    const int R = h->R;
    std::vector<Seg> hs = {Seg{0, 0, 0}, Seg{0, 1, 0}, Seg{1, 0, 0}, Seg{1, 1, 0}};
    std::vector<Tile> ht;
    add_tiles(ht, 0, (int)h->n, {2, 3}, R, h->d_OT, 2 * R);   // O' x [T' | E T' + U]
    add_tiles(ht, 1, (int)h->n, {2}, R, h->d_XT, R);          // X' x T'
    add_tiles(ht, 2, R, {2, 3}, R, h->d_TT, 2 * R);           // T' x [T' | E T' + U]
    h->nsegh = (int)hs.size();
    h->ntileh = (int)ht.size();
    if (s == BLM_OK) s = upload(h, hs, &h->d_segh);
    if (s == BLM_OK) s = upload(h, ht, &h->d_tileh);
  }
  {
    std::vector<Seg> cs = {Seg{1, 0, 0}, Seg{1, 1, 0}};       // p, E p + r
    std::vector<Tile> ct;
    add_tiles(ct, 0, (int)h->dc, {0, 1}, (int)h->dc, h->d_Cc, 2 * h->dc);
    h->nsegc = (int)cs.size();
    h->ntilec = (int)ct.size();
    if (s == BLM_OK) s = upload(h, cs, &h->d_segc);
    if (s == BLM_OK) s = upload(h, ct, &h->d_tilec);
  }
  {
    std::vector<ProjBlock> pbB(h->nb), pbD(h->nb);
    std::vector<BlockAsm> ba(h->nb);
    std::vector<EigProblem> ep(h->nb);
    std::vector<DirBlock> dbk(h->nb);
    for (int b = 0; b < h->nb; ++b) {
      const int64_t D = h->db[b] + 1;
      pbB[b] = ProjBlock{h->off[b], h->Mb[b], h->Kb[b], h->oc[b], 0, h->d_B + h->B_off[b], h->Mb[b],
                         h->d_B32 + h->B_off[b]};
      pbD[b] = ProjBlock{h->off[b], h->Mb[b], h->n_old, b * h->n_old, 0,
                         h->d_D ? h->d_D + h->off[b] : nullptr, h->n, nullptr};
      ba[b] = BlockAsm{h->off[b], h->Mb[b], h->db[b], b, 0, h->d_C + h->C_off[b],
                       h->d_S + h->SH_off[b], h->d_H + h->SH_off[b]};
      ep[b] = EigProblem{(int)D, h->Kb[b], 0, 0, h->d_S + h->SH_off[b], h->d_H + h->SH_off[b],
                         h->d_eigw + h->eigw_off[b], h->d_lam + h->lam_off[b],
                         h->d_evec + h->vec_off[b], h->d_status + b};
      dbk[b] = DirBlock{h->Mb[b], h->Kb[b], (int)D, 0, h->d_evec + h->vec_off[b],
                        h->d_B + h->B_off[b], h->d_status + b};
    }
    std::vector<EigProblem> cp(1);
    cp[0] = EigProblem{(int)(h->dc + 1), 1, 1, 0, h->d_Sc, h->d_Hc, h->d_ceigw, h->d_clam,
                       h->d_cev, h->d_status + h->nb};
    if (s == BLM_OK) s = upload(h, pbB, &h->d_pbB);
    if (s == BLM_OK) s = upload(h, pbD, &h->d_pbD);
    if (s == BLM_OK) s = upload(h, ba, &h->d_asm);
    if (s == BLM_OK) s = upload(h, ep, &h->d_eigp);
    if (s == BLM_OK) s = upload(h, dbk, &h->d_dirb);
    if (s == BLM_OK) s = upload(h, cp, &h->d_ceigp);
  }
  if (s == BLM_OK && h->prec != BLM_PREC_F64) {
    // tensor-core tiles: 128 rows x 256 columns of [Y'Y'^T | Y'(E Y' + Z)^T] per block, and the
    // same over the combined directions (one block of dc columns of the projection scratch)
    std::vector<TcTile> t1, t2;
    // column tiles never straddle the Y' | X' boundary: Y' tiles start at 0, 256, .. < m and
    // X' tiles at m, m + 256, .. < 2m
    auto add = [](std::vector<TcTile>& v, int64_t lo, int m, double* out) {
      for (int r0 = 0; r0 < m; r0 += 128) {
        for (int c0 = 0; c0 < m; c0 += 256) v.push_back(TcTile{lo, m, r0, c0, 0, out});
        for (int c0 = m; c0 < 2 * m; c0 += 256) v.push_back(TcTile{lo, m, r0, c0, 0, out});
      }
    };
    for (int b = 0; b < h->nb; ++b) add(t1, h->off[b], h->Mb[b], h->d_C + h->C_off[b]);
    add(t2, 0, (int)h->dc, h->d_Cc);
    // the combined overlap is symmetric and assembled from its upper triangle: overlap tiles
    // wholly below the diagonal (last column < first row) are not computed
    t2.erase(std::remove_if(t2.begin(), t2.end(),
                            [](const TcTile& t) { return t.col0 < t.m && t.col0 + 256 <= t.row0; }),
             t2.end());
    h->ntc1 = (int)t1.size();
    h->ntc2 = (int)t2.size();
    s = upload(h, t1, &h->d_tc1);
    if (s == BLM_OK) s = upload(h, t2, &h->d_tc2);
  }
  if (s == BLM_OK) s = zero_sums(h);
  if (s == BLM_OK && h->n_old > 0) {
    BLM_CU(h, cudaMemsetAsync(h->d_hgram, 0, 8 * (size_t)h->R * h->R, h->st));
    launch_gram(h->d_pbD, h->nb, h->n_old, h->d_hgram, h->R, h->st);
  }
  if (s == BLM_OK) {
    e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) s = cuda_fail(h, e, "blm_create");
  }
  if (s != BLM_OK) {
    fprintf(stderr, "blm_create: %s\n", h->err.c_str());
    blm_destroy(h);
    return s;
  }
  *out = h;
  return BLM_OK;
}

blm_status blm_accumulate(blm_handle* h, const void* O, const void* dEL, const void* EL,
                          const void* w, int64_t n_samples, int64_t ld) {
  if (!h) return BLM_ERR_ARG;
  if (h->state != ST_CREATED && h->state != ST_ACCUM)
    return fail(h, BLM_ERR_STATE, "blm_accumulate after blm_block_solve (call blm_reset)");
  if (n_samples < 0 || ld < h->n) return fail(h, BLM_ERR_ARG, "bad n_samples or ld");
  if (n_samples == 0) return BLM_OK;
  if (!O || !dEL || !EL) return fail(h, BLM_ERR_ARG, "NULL sample array");
  blm_status s = h->in_type == BLM_IN_F64
                     ? sweep<double>(h, 1, O, dEL, EL, w, n_samples, ld)
                     : sweep<float>(h, 1, O, dEL, EL, w, n_samples, ld);
  if (s != BLM_OK) return s;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "blm_accumulate");
  h->state = ST_ACCUM;
  return BLM_OK;
}

blm_status blm_block_solve(blm_handle* h) {
  if (!h) return BLM_ERR_ARG;
  if (h->state != ST_ACCUM) return fail(h, BLM_ERR_STATE, "blm_block_solve needs accumulated samples");
  cudaStream_t st = h->st;
  HistSums hs{h->n_old, h->nb, h->d_OT, h->d_XT, h->d_TT, h->d_hvec,
              h->d_hvec ? h->d_hvec + h->R : nullptr, h->d_hvec ? h->d_hvec + 2 * h->R : nullptr,
              h->d_hgram};
  BLM_CU(h, cudaMemsetAsync(h->d_status, 0, 4 * (h->nb + 2), st));
  {
    Prof pr(h, PC_ASSEMBLE);
    launch_assemble_blocks(h->d_asm, h->nb, h->maxD, h->d_vec, h->d_vec + h->n,
                           h->d_vec + 2 * h->n, h->d_scal, hs, h->shift, st);
  }
  {
    Prof pr(h, PC_EIG_BLOCKS);
    launch_eig(h->d_eigp, h->nb, 512, st);
  }
  {
    Prof pr(h, PC_DIRS, h->shift != 0.0 ? 3 : 2);
    launch_extract_dirs(h->d_dirb, h->nb, st);
    if (h->in_type == BLM_IN_F32) launch_to_f32(h->d_B, h->d_B32, h->B_words, st);
    launch_cen(h->d_pbB, h->nb, h->d_vec, h->d_scal, h->d_cen, st);
    if (h->shift != 0.0) {
      BLM_CU(h, cudaMemsetAsync(h->d_cgram, 0, 8 * h->dc * h->dc, st));
      launch_gram(h->d_pbB, h->nb, h->maxK, h->d_cgram, h->dc, st);
    }
  }
  std::vector<int32_t> stat(h->nb + 3);
  BLM_CU(h, cudaMemcpyAsync(stat.data(), h->d_status, 4 * (h->nb + 3), cudaMemcpyDeviceToHost, st));
  BLM_CU(h, cudaStreamSynchronize(st));
  BLM_CU(h, cudaGetLastError());
  if (stat[h->nb + 2] != 0) {
    char buf[160];
    snprintf(buf, sizeof buf, "tensor-core sweep: a bounded wait ran out (code %d)", stat[h->nb + 2]);
    return fail(h, BLM_ERR_TIMEOUT, buf);
  }
  for (int b = 0; b < h->nb; ++b)
    if (stat[b] != ST_OK) {
      char buf[160];
      snprintf(buf, sizeof buf, "block %d: %s", b, status_text(stat[b]));
      return fail(h, BLM_ERR_NUMERIC, buf);
    }
  h->state = ST_BLOCKS;
  return BLM_OK;
}

blm_status blm_project(blm_handle* h, const void* O, const void* dEL, const void* EL,
                       const void* w, int64_t n_samples, int64_t ld) {
  if (!h) return BLM_ERR_ARG;
  if (h->state != ST_BLOCKS && h->state != ST_PROJ)
    return fail(h, BLM_ERR_STATE, "blm_project needs blm_block_solve first");
  if (n_samples < 0 || ld < h->n) return fail(h, BLM_ERR_ARG, "bad n_samples or ld");
  if (n_samples == 0) return BLM_OK;
  if (!O || !dEL || !EL) return fail(h, BLM_ERR_ARG, "NULL sample array");
  blm_status s = h->in_type == BLM_IN_F64
                     ? sweep<double>(h, 2, O, dEL, EL, w, n_samples, ld)
                     : sweep<float>(h, 2, O, dEL, EL, w, n_samples, ld);
  if (s != BLM_OK) return s;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "blm_project");
  h->state = ST_PROJ;
  return BLM_OK;
}

blm_status blm_combined_solve(blm_handle* h, double* dmu, double* e_pred) {
  if (!h) return BLM_ERR_ARG;
  if (h->state != ST_PROJ) return fail(h, BLM_ERR_STATE, "blm_combined_solve needs blm_project first");
  if (!dmu || !e_pred) return fail(h, BLM_ERR_ARG, "NULL output");
  cudaStream_t st = h->st;
  {
    Prof pr(h, PC_ASSEMBLE);
    launch_assemble_combined(h->dc, h->d_Cc, h->d_cvec, h->d_cvec + h->dc,
                             h->d_cvec + 2 * h->dc, h->d_scal,
                             h->shift != 0.0 ? h->d_cgram : nullptr, h->shift, h->d_Sc, h->d_Hc, st);
  }
  {
    Prof pr(h, PC_EIG_COMBINED);
    if (h->dc + 1 <= kDenseCombinedMax) {
      launch_eig(h->d_ceigp, 1, 512, st);
    } else {
      launch_davidson(h->d_ceigp, 1, kDavidsonTol, kDavidsonIter, st);
      // a Davidson run that did not converge (clustered or ill-conditioned combined problems
      // from few samples) falls back to the dense solver on the same matrices
      int32_t dstat = 0;
      BLM_CU(h, cudaMemcpyAsync(&dstat, h->d_status + h->nb, 4, cudaMemcpyDeviceToHost, st));
      BLM_CU(h, cudaStreamSynchronize(st));
      if (dstat == ST_NOCONV) launch_eig(h->d_ceigp, 1, 512, st);
    }
  }
  {
    Prof pr(h, PC_UPDATE, 2);
    launch_update(h->nb, h->d_pbB, h->dc, h->d_cev, h->d_shift, h->d_vec, h->d_scal,
                  h->d_scal + 3, h->d_dmu, h->d_status + h->nb + 1, st);
  }
  int32_t stat[3];
  double lam;
  BLM_CU(h, cudaMemcpyAsync(stat, h->d_status + h->nb, 12, cudaMemcpyDeviceToHost, st));
  BLM_CU(h, cudaMemcpyAsync(&lam, h->d_clam, 8, cudaMemcpyDeviceToHost, st));
  BLM_CU(h, cudaMemcpyAsync(dmu, h->d_dmu, 8 * h->n, cudaMemcpyDefault, st));
  BLM_CU(h, cudaStreamSynchronize(st));
  BLM_CU(h, cudaGetLastError());
  if (stat[2] != 0) return fail(h, BLM_ERR_TIMEOUT, "tensor-core sweep: a bounded wait ran out");
  if (stat[0] != ST_OK) return fail(h, BLM_ERR_NUMERIC, std::string("combined: ") + status_text(stat[0]));
  if (stat[1] != ST_OK) return fail(h, BLM_ERR_NUMERIC, std::string("update: ") + status_text(stat[1]));
  *e_pred = lam;
  h->state = ST_DONE;
  return BLM_OK;
}

blm_status blm_get_block(blm_handle* h, int32_t b, double* S, double* H, double* lambda,
                         double* B) {
  if (!h) return BLM_ERR_ARG;
  if (b < 0 || b >= h->nb) return fail(h, BLM_ERR_ARG, "block index out of range");
  if (h->state < ST_BLOCKS) return fail(h, BLM_ERR_STATE, "blocks not solved yet");
  const int64_t D = h->db[b] + 1;
  if (S) BLM_CU(h, cudaMemcpyAsync(S, h->d_S + h->SH_off[b], 8 * D * D, cudaMemcpyDefault, h->st));
  if (H) BLM_CU(h, cudaMemcpyAsync(H, h->d_H + h->SH_off[b], 8 * D * D, cudaMemcpyDefault, h->st));
  if (lambda) BLM_CU(h, cudaMemcpyAsync(lambda, h->d_lam + h->lam_off[b], 8 * h->Kb[b], cudaMemcpyDefault, h->st));
  if (B) BLM_CU(h, cudaMemcpyAsync(B, h->d_B + h->B_off[b], 8 * (int64_t)h->Kb[b] * h->Mb[b], cudaMemcpyDefault, h->st));
  BLM_CU(h, cudaStreamSynchronize(h->st));
  return BLM_OK;
}

blm_status blm_get_combined(blm_handle* h, double* S, double* H) {
  if (!h) return BLM_ERR_ARG;
  if (h->state < ST_DONE) return fail(h, BLM_ERR_STATE, "combined problem not solved yet");
  const int64_t D = h->dc + 1;
  if (S) BLM_CU(h, cudaMemcpyAsync(S, h->d_Sc, 8 * D * D, cudaMemcpyDefault, h->st));
  if (H) BLM_CU(h, cudaMemcpyAsync(H, h->d_Hc, 8 * D * D, cudaMemcpyDefault, h->st));
  BLM_CU(h, cudaStreamSynchronize(h->st));
  return BLM_OK;
}

int64_t blm_block_dim(const blm_handle* h, int32_t b) {
  if (!h || b < 0 || b >= h->nb) return -1;
  return h->db[b];
}

int64_t blm_combined_dim(const blm_handle* h) { return h ? h->dc : -1; }

blm_status blm_reset(blm_handle* h) {
  if (!h) return BLM_ERR_ARG;
  return zero_sums(h);
}

blm_status blm_destroy(blm_handle* h) {
  if (!h) return BLM_OK;
  cudaFree(h->base);
  void* tabs[] = {h->d_seg1, h->d_tile1, h->d_segh, h->d_tileh, h->d_segc, h->d_tilec,
                  h->d_pbB, h->d_pbD, h->d_asm, h->d_eigp, h->d_ceigp, h->d_dirb, h->d_tc1,
                  h->d_tc2};
  for (void* p : tabs)
    if (p) cudaFree(p);
  for (int b = 0; b < 2; ++b) {
    for (int k = 0; k < 4; ++k)
      if (h->d_stage[b][k]) cudaFree(h->d_stage[b][k]);
    if (h->ev_copy[b]) cudaEventDestroy(h->ev_copy[b]);
    if (h->ev_done[b]) cudaEventDestroy(h->ev_done[b]);
  }
  if (h->copy_st) cudaStreamDestroy(h->copy_st);
  for (auto& pe : h->prof_ev) {
    cudaEventDestroy(pe.second.first);
    cudaEventDestroy(pe.second.second);
  }
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  delete h;
  return BLM_OK;
}

const char* blm_last_error(const blm_handle* h) { return h ? h->err.c_str() : "NULL handle"; }

blm_status blm_profile(blm_handle* h, int enable) {
  if (!h) return BLM_ERR_ARG;
  BLM_CU(h, cudaStreamSynchronize(h->st));
  for (auto& pe : h->prof_ev) {
    h->ev_pool.push_back(pe.second.first);
    h->ev_pool.push_back(pe.second.second);
  }
  h->prof_ev.clear();
  for (int i = 0; i < BLM_PROF_CLASSES; ++i) h->prof_launch[i] = 0;
  h->prof = enable != 0;
  return BLM_OK;
}

blm_status blm_profile_read(blm_handle* h, int n, double* ms, int64_t* launches) {
  if (!h || n < 0 || n > BLM_PROF_CLASSES) return BLM_ERR_ARG;
  BLM_CU(h, cudaStreamSynchronize(h->st));
  std::vector<double> acc(BLM_PROF_CLASSES, 0.0);
  for (auto& pe : h->prof_ev) {
    float t = 0.0f;
    BLM_CU(h, cudaEventElapsedTime(&t, pe.second.first, pe.second.second));
    acc[pe.first] += t;
  }
  for (int i = 0; i < n; ++i) {
    if (ms) ms[i] = acc[i];
    if (launches) launches[i] = h->prof_launch[i];
  }
  return BLM_OK;
}

const char* blm_profile_class_name(int i) {
  return (i >= 0 && i < BLM_PROF_CLASSES) ? kProfNames[i] : "";
}

}  // extern "C"
