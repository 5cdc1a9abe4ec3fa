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

constexpr int64_t kSubChunk = 65536;     // default samples per scratch pass (operands, projections)
constexpr int64_t kShiftSamples = 65536; // samples that fix the reference shift
constexpr int64_t kStagePiece = 32768;   // samples per host-to-device copy of host sample arrays
// Combined problems up to this dimension use the dense solver (exact ordering of the whole
// spectrum); larger ones use generalized Davidson for the lowest eigenpair.
constexpr int64_t kDenseCombinedMax = 320;
constexpr double kDavidsonTol = 1e-13;
constexpr int kDavidsonIter = 400;

struct Alloc {
  // offsets in bytes of every device buffer in the handle's one allocation; filled by plan().
  // Buffers of 64 MiB and more start on 2 MiB boundaries (the large-page size), the rest on 256 B.
  size_t total = 0;
  std::vector<std::pair<void**, size_t>> items;
  void add(void** p, size_t bytes) {
    const size_t align = bytes >= ((size_t)64 << 20) ? ((size_t)2 << 20) : 256;
    total = (total + align - 1) / align * align;
    items.emplace_back(p, total);
    total += (bytes + 255) / 256 * 256;
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
  uint32_t wait_limit = BLM_WAIT_LIMIT_DEFAULT;   // tensor-core pipeline waits: polls
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
  int64_t sub_chunk = kSubChunk;            // samples per scratch pass
  uint8_t* d_opA = nullptr;                 // prepared split operands of a sub-chunk:
  uint8_t* d_opBS = nullptr;                //   Y', w Y', w X' rows (n of them; dc in the
  uint8_t* d_opBH = nullptr;                //   second sweep)
  uint8_t* d_opT[3] = {nullptr, nullptr, nullptr};   // history: T', w T', w (E T' + U) (R rows)
  float* d_D32 = nullptr;                   // history directions in FP32 (split precisions)
  int64_t op_row_bytes = 0;                 //   bytes per parameter row (128 per sample group)
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
  void* d_scrY = nullptr;        // sub_chunk x max(R, dc)
  void* d_scrZ = nullptr;
  double* d_S = nullptr;         // block S matrices
  double* d_H = nullptr;
  double* d_eigw = nullptr;
  std::vector<int32_t> eig_dims;           // block problem dimensions (team sizes of the solver)
  int32_t cdim = 0;                        // combined problem dimension
  void* d_teamctl = nullptr;               // team control blocks: nb block problems
  void* d_cteamctl = nullptr;              // and the combined problem
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
  EigProblem* d_ceigp = nullptr;            // [0] the combined problem, [1] its dense fallback
                                            //     (runs only if Davidson reports ST_NOCONV)
  DirBlock* d_dirb = nullptr;
  TcTile* d_tc1 = nullptr;  int ntc1 = 0;   // pass-1 tensor-core tiles (the chosen layout)
  TcTile* d_tc2 = nullptr;  int ntc2 = 0;   // combined tensor-core tiles
  TcTile* d_tc1_layout[2] = {nullptr, nullptr};   // per-block tiles, packed band tiles
  int ntc1_layout[2] = {0, 0};
  int layout = 0;                           // pass-1 tile layout in use (blm_autotune)
  int64_t tc_range_max = 16384;             // longest work-unit sample range (blm_autotune)
  int32_t* d_blk_of = nullptr;              // packed tiles: block of each parameter,
  int64_t* d_blk_lo = nullptr;              //   block offsets, sizes and sums
  int32_t* d_blk_m = nullptr;
  double** d_blk_C = nullptr;
  int off_aligned = 0;                     // block offsets all multiples of 4
  // host staging
  void* d_stage[2][4] = {{nullptr}};
  int64_t stage_rows = 0;
  // device copies of host sample pieces kept from the first sweep for the second
  // (blm_set_host_cache): key = host address of the piece's O rows, its G rows, row count, ld
  struct CachedPiece {
    const void* O;
    const void* G;
    int64_t rows, ld;
    void* d[4];
  };
  char* hc_pool = nullptr;
  size_t hc_capacity = 0, hc_used = 0;
  std::vector<CachedPiece> hc_pieces;
  cudaStream_t copy_st = nullptr;
  cudaEvent_t ev_copy[2] = {nullptr, nullptr};
  cudaEvent_t ev_done[2] = {nullptr, nullptr};
  void* base = nullptr;   // single device allocation
  // captured step (blm_graph_capture)
  cudaStream_t graph_st = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  // profiling
  bool prof = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_ev;
  std::vector<cudaEvent_t> ev_pool;
  int64_t prof_launch[BLM_PROF_CLASSES] = {0};
};

// A batch of independent optimisations (blm_batch_*): one handle per problem, one graph.
struct blm_batch {
  std::vector<blm_handle*> hs;
  cudaStream_t st = nullptr;              // the caller's stream: launches and results
  cudaStream_t cap_st = nullptr;          // origin stream of the capture
  std::vector<cudaEvent_t> ev;            // per problem: joins of its branch
  cudaEvent_t ev_fork = nullptr;
  EigProblem* d_blocks = nullptr;         // every problem's block problems, one launch
  int nblocks_all = 0;
  EigProblem* d_comb = nullptr;           // the dense combined problems, one launch
  int ncomb_dense = 0;
  std::vector<int32_t> blk_dims, comb_dims;   // their dimensions (team sizes)
  void* d_teamctl = nullptr;              // team control blocks of both launches
  cudaGraphExec_t exec = nullptr;
  std::string err;
};

namespace {

enum ProfClass {
  PC_SHIFT = 0, PC_SUMS = 1, PC_CONTRACT = 2, PC_TC1 = 3, PC_HIST = 4, PC_ASSEMBLE = 5,
  PC_EIG_BLOCKS = 6, PC_DIRS = 7, PC_PROJECT = 8, PC_TC2 = 9, PC_EIG_COMBINED = 10, PC_UPDATE = 11,
  PC_PREP = 12, PC_PREP2 = 13
};
const char* kProfNames[BLM_PROF_CLASSES] = {
    "reference_shift", "first_moments", "contract_f64", "contract_tc_pass1", "history_terms",
    "assemble", "eig_blocks", "directions", "project", "contract_tc_pass2", "eig_combined",
    "update", "operand_prep_pass1", "operand_prep_pass2"};

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
      p->precision != BLM_PREC_TF32X4) {
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
  if (!(p->shift >= 0.0) || !isfinite(p->shift)) { why = "shift must be finite and >= 0"; return BLM_ERR_ARG; }
  if (p->pass_samples != 0 &&
      (p->pass_samples < 1024 || p->pass_samples > (1 << 20) || p->pass_samples % 1024 != 0)) {
    why = "pass_samples must be 0 or a multiple of 1024 in 1024 .. 2^20";
    return BLM_ERR_ARG;
  }
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
  h->sub_chunk = p->pass_samples ? p->pass_samples : kSubChunk;
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
  a.add((void**)&h->d_scrY, h->selem * h->sub_chunk * scr_cols);
  a.add((void**)&h->d_scrZ, h->selem * h->sub_chunk * scr_cols);
  a.add((void**)&h->d_S, 8 * SHsz);
  a.add((void**)&h->d_H, 8 * SHsz);
  a.add((void**)&h->d_eigw, 8 * EWsz);
  a.add((void**)&h->d_teamctl, eig_team_ctl_bytes(h->nb));
  a.add((void**)&h->d_cteamctl, eig_team_ctl_bytes(1));
  a.add((void**)&h->d_lam, 8 * LOsz);
  a.add((void**)&h->d_evec, 8 * VOsz);
  a.add((void**)&h->d_B, 8 * BOsz);
  a.add((void**)&h->d_B32, 4 * BOsz);
  if (h->prec != BLM_PREC_F64) {
    // 128 bytes per 32 samples (BF16 hi + lo) or per 16 samples (TF32 hi + lo)
    h->op_row_bytes = h->sub_chunk / (h->prec == BLM_PREC_TF32X4 ? 16 : 32) * 128;
    // (staggered: the arrays the preparation writes together must not start a power-of-two
    // distance apart -- with 4 GiB arrays back to back the first sweep's preparation took
    // 52.9 ms per step, with these 3 and 5 MiB gaps 44.4 ms)
    a.add((void**)&h->d_opA, h->op_row_bytes * n + ((size_t)3 << 20));
    a.add((void**)&h->d_opBS, h->op_row_bytes * n + ((size_t)5 << 20));
    a.add((void**)&h->d_opBH, h->op_row_bytes * n);
    if (h->n_old > 0) {
      for (int k = 0; k < 3; ++k) a.add((void**)&h->d_opT[k], h->op_row_bytes * h->R);
      a.add((void**)&h->d_D32, 4 * h->n_old * n);
    }
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
  h->hc_used = 0;
  h->hc_pieces.clear();
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
TcPack pack_tables(const blm_handle* h) {
  return TcPack{h->d_blk_of, h->d_blk_lo, h->d_blk_m, h->d_blk_C};
}

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
      for (int64_t s0 = 0; s0 < ns; s0 += h->sub_chunk) {
        const int64_t cnt = std::min(h->sub_chunk, ns - s0);
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
  } else {
    // split precision: operands prepared once per element, then TMA + tensor cores; with
    // history directions the projections t = O'_k . D_jk, u = G_k . D_jk are prepared too and
    // their sums with the block rows (Eq. 10) are further tiles of the same launch
    const int tf = h->prec == BLM_PREC_TF32X4;
    for (int64_t s0 = 0; s0 < ns; s0 += h->sub_chunk) {
      const int64_t cnt = std::min(h->sub_chunk, ns - s0);
      const float* Os = (const float*)O + s0 * ld;
      const float* Gs = (const float*)G + s0 * ld;
      const float* Es = (const float*)E + s0;
      const float* Wp = w ? (const float*)w + s0 : nullptr;
      {
        Prof pr(h, PC_PREP);
        launch_prep(Os, Gs, Es, Wp, cnt, ld, h->n, h->d_shift32, h->d_opA, h->d_opBS, h->d_opBH,
                    h->op_row_bytes, h->d_vec, h->d_vec + h->n, h->d_vec + 2 * h->n, h->d_scal, tf,
                    st);
      }
      TcOperands ops{};
      ops.op[0] = h->d_opA;
      ops.op[1] = Wp ? h->d_opBS : h->d_opA;
      ops.op[2] = h->d_opBH;
      ops.rows[0] = ops.rows[1] = ops.rows[2] = h->n;
      if (h->n_old > 0) {
        const int64_t R = h->R;
        float* TY = (float*)h->d_scrY;
        float* TZ = (float*)h->d_scrZ;
        Prof pr(h, PC_HIST, 2);
        if (!launch_project_rb(Os, Gs, ld, h->d_shift32, h->d_pbD, h->nb, h->off_aligned != 0,
                               nullptr, TY, TZ, R, cnt, h->n_old, st))
          launch_project<float, float>(Os, Gs, ld, ld, h->d_shift, h->d_shift32, h->d_pbD, h->nb,
                                       nullptr, TY, TZ, R, cnt, h->maxM, h->n_old, st);
        launch_prep(TY, TZ, Es, Wp, cnt, R, R, nullptr, h->d_opT[0], h->d_opT[1], h->d_opT[2],
                    h->op_row_bytes, h->d_hvec, h->d_hvec + R, h->d_hvec + 2 * R, nullptr, tf, st);
        ops.op[3] = h->d_opT[0];
        ops.op[4] = Wp ? h->d_opT[1] : h->d_opT[0];
        ops.op[5] = h->d_opT[2];
        ops.rows[3] = ops.rows[4] = ops.rows[5] = R;
      }
      Prof pr(h, PC_TC1);
      cudaError_t e = launch_tc_prepared(ops, h->op_row_bytes, cnt, h->d_tc1, h->ntc1,
                                         Wp != nullptr, h->d_status + h->nb + 2, h->wait_limit,
                                         tf, pack_tables(h), h->tc_range_max, st);
      if (e != cudaSuccess) return cuda_fail(h, e, "launch_tc_prepared");
    }
  }
  return BLM_OK;
}

template <typename T>
blm_status project_dev(blm_handle* h, const T* O, const T* G, const T* E, const T* w,
                       int64_t ns, int64_t ld) {
  cudaStream_t st = h->st;
  const int64_t dc = h->dc;
  for (int64_t s0 = 0; s0 < ns; s0 += h->sub_chunk) {
    const int64_t cnt = std::min(h->sub_chunk, ns - s0);
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
      // split-precision paths (FP32 inputs only): the projections p (centred) and r, then the
      // first sweep's route -- prepared operands (no shift), TMA + tensor cores
      float* PY = (float*)h->d_scrY;
      float* PZ = (float*)h->d_scrZ;
      const int tf = h->prec == BLM_PREC_TF32X4;
      {
        Prof pr(h, PC_PROJECT);
        if (!launch_project_rb(Os, Gs, ld, h->d_shift ? h->d_shift32 : nullptr, h->d_pbB, h->nb,
                               h->off_aligned != 0, h->d_cen, PY, PZ, dc, cnt, h->maxK, st))
          launch_project<float, float>(Os, Gs, ld, ld, h->d_shift, h->d_shift32, h->d_pbB, h->nb,
                                       h->d_cen, PY, PZ, dc, cnt, h->maxM, h->maxK, st);
      }
      {
        Prof pr(h, PC_PREP2);
        launch_prep(PY, PZ, Es, ws, cnt, dc, dc, nullptr, h->d_opA, h->d_opBS, h->d_opBH,
                    h->op_row_bytes, h->d_cvec, h->d_cvec + dc, h->d_cvec + 2 * dc, nullptr, tf,
                    st);
      }
      TcOperands ops{};
      ops.op[0] = h->d_opA;
      ops.op[1] = ws ? h->d_opBS : h->d_opA;
      ops.op[2] = h->d_opBH;
      ops.rows[0] = ops.rows[1] = ops.rows[2] = dc;
      Prof pr(h, PC_TC2);
      cudaError_t e = launch_tc_prepared(ops, h->op_row_bytes, cnt, h->d_tc2, h->ntc2,
                                         ws != nullptr, h->d_status + h->nb + 2, h->wait_limit,
                                         tf, pack_tables(h), h->tc_range_max, st);
      if (e != cudaSuccess) return cuda_fail(h, e, "launch_tc_prepared (combined)");
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
  // host memory: stage through two device buffers, or (first sweep, with a host cache) copy
  // into the cache and keep the copy for the second sweep
  const size_t es = sizeof(T);
  if (!h->d_stage[0][0]) {
    // pieces of up to kStagePiece samples: large enough that each piece's tensor-core launch
    // keeps every SM busy (the copies, at the host link's rate, bound the step either way)
    int64_t rows = std::min<int64_t>(kStagePiece, ns);
    rows = std::max<int64_t>(rows, std::min<int64_t>(kStagePiece, 4096));
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
  for (int64_t s0 = 0; s0 < ns; s0 += rows) {
    const int64_t cnt = std::min(rows, ns - s0);
    const char* hO = (const char*)O + s0 * ld * es;
    const char* hG = (const char*)G + s0 * ld * es;
    // second sweep: a piece the first sweep left in the cache needs no copy
    const blm_handle::CachedPiece* hit = nullptr;
    if (pass == 2)
      for (const auto& cp : h->hc_pieces)
        if (cp.O == hO && cp.G == hG && cp.rows == cnt && cp.ld == ld) {
          hit = &cp;
          break;
        }
    if (hit) {
      const T* dw = w ? (const T*)hit->d[3] : nullptr;
      blm_status st2 = project_dev<T>(h, (const T*)hit->d[0], (const T*)hit->d[1],
                                      (const T*)hit->d[2], dw, cnt, h->n);
      if (st2 != BLM_OK) return st2;
      continue;
    }
    // a cached piece holds O, G (cnt x n each), E and w (cnt each), each 256-byte aligned
    const size_t a_rows = (es * (size_t)cnt * h->n + 255) / 256 * 256;
    const size_t a_vec = (es * (size_t)cnt + 255) / 256 * 256;
    const size_t piece_bytes = 2 * a_rows + 2 * a_vec;
    void* dst[4];
    bool cached = false;
    if (pass == 1 && h->hc_pool && h->hc_used + piece_bytes <= h->hc_capacity) {
      char* p = h->hc_pool + h->hc_used;
      dst[0] = p;
      dst[1] = p + a_rows;
      dst[2] = p + 2 * a_rows;
      dst[3] = p + 2 * a_rows + a_vec;
      h->hc_used += piece_bytes;
      h->hc_pieces.push_back(blm_handle::CachedPiece{hO, hG, cnt, ld, {dst[0], dst[1], dst[2], dst[3]}});
      cached = true;
    } else {
      for (int k = 0; k < 4; ++k) dst[k] = h->d_stage[buf][k];
      BLM_CU(h, cudaStreamWaitEvent(h->copy_st, h->ev_done[buf], 0));
    }
    if (ld == h->n) {   // contiguous rows: one linear copy per array
      BLM_CU(h, cudaMemcpyAsync(dst[0], hO, es * h->n * cnt, cudaMemcpyHostToDevice, h->copy_st));
      BLM_CU(h, cudaMemcpyAsync(dst[1], hG, es * h->n * cnt, cudaMemcpyHostToDevice, h->copy_st));
    } else {
      BLM_CU(h, cudaMemcpy2DAsync(dst[0], es * h->n, hO, es * ld, es * h->n, cnt,
                                  cudaMemcpyHostToDevice, h->copy_st));
      BLM_CU(h, cudaMemcpy2DAsync(dst[1], es * h->n, hG, es * ld, es * h->n, cnt,
                                  cudaMemcpyHostToDevice, h->copy_st));
    }
    BLM_CU(h, cudaMemcpyAsync(dst[2], (const char*)E + s0 * es, es * cnt,
                              cudaMemcpyHostToDevice, h->copy_st));
    if (w)
      BLM_CU(h, cudaMemcpyAsync(dst[3], (const char*)w + s0 * es, es * cnt,
                                cudaMemcpyHostToDevice, h->copy_st));
    BLM_CU(h, cudaEventRecord(h->ev_copy[buf], h->copy_st));
    BLM_CU(h, cudaStreamWaitEvent(h->st, h->ev_copy[buf], 0));
    const T* dO = (const T*)dst[0];
    const T* dG = (const T*)dst[1];
    const T* dE = (const T*)dst[2];
    const T* dw = w ? (const T*)dst[3] : nullptr;
    blm_status s = pass == 1 ? accumulate_dev<T>(h, dO, dG, dE, dw, cnt, h->n)
                             : project_dev<T>(h, dO, dG, dE, dw, cnt, h->n);
    if (s != BLM_OK) return s;
    if (!cached) BLM_CU(h, cudaEventRecord(h->ev_done[buf], h->st));
    buf ^= 1;
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

// Block assembly, eigen-solves, directions: launches only (stream-ordered, capturable).  The
// three phases are separate so that a batch can solve every problem's blocks in one launch.
blm_status block_solve_pre(blm_handle* h) {
  cudaStream_t st = h->st;
  HistSums hs{h->n_old, h->nb, h->d_OT, h->d_XT, h->d_TT, h->d_hvec,
              h->d_hvec ? h->d_hvec + h->R : nullptr, h->d_hvec ? h->d_hvec + 2 * h->R : nullptr,
              h->d_hgram};
  BLM_CU(h, cudaMemsetAsync(h->d_status, 0, 4 * (h->nb + 2), st));
  Prof pr(h, PC_ASSEMBLE);
  launch_assemble_blocks(h->d_asm, h->nb, h->maxD, h->d_vec, h->d_vec + h->n,
                         h->d_vec + 2 * h->n, h->d_scal, hs, h->shift, st);
  return BLM_OK;
}

blm_status block_solve_post(blm_handle* h) {
  cudaStream_t st = h->st;
  Prof pr(h, PC_DIRS, h->shift != 0.0 ? 3 : 2);
  launch_extract_dirs(h->d_dirb, h->nb, st);
  if (h->in_type == BLM_IN_F32) launch_to_f32(h->d_B, h->d_B32, h->B_words, st);
  launch_cen(h->d_pbB, h->nb, h->d_vec, h->d_scal, h->d_cen, st);
  if (h->shift != 0.0) {
    BLM_CU(h, cudaMemsetAsync(h->d_cgram, 0, 8 * h->dc * h->dc, st));
    launch_gram(h->d_pbB, h->nb, h->maxK, h->d_cgram, h->dc, st);
  }
  return BLM_OK;
}

blm_status enqueue_block_solve(blm_handle* h) {
  blm_status s = block_solve_pre(h);
  if (s != BLM_OK) return s;
  {
    Prof pr(h, PC_EIG_BLOCKS);
    launch_eig(h->d_eigp, h->nb, 512, h->st, h->eig_dims.data(), h->d_teamctl);
  }
  s = block_solve_post(h);
  if (s != BLM_OK) return s;
  BLM_CU(h, cudaGetLastError());
  return BLM_OK;
}

// Reads the status words of the first sweep and the block solves (synchronises the stream).
blm_status block_status(blm_handle* h) {
  std::vector<int32_t> stat(h->nb + 3);
  BLM_CU(h, cudaMemcpyAsync(stat.data(), h->d_status, 4 * (h->nb + 3), cudaMemcpyDeviceToHost, h->st));
  BLM_CU(h, cudaStreamSynchronize(h->st));
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
  return BLM_OK;
}

// Combined assembly, lowest eigenpair and update: launches only (capturable).  Davidson's dense
// fallback is decided on the device.  dmu may be host memory only outside a capture.
blm_status combined_pre(blm_handle* h) {
  Prof pr(h, PC_ASSEMBLE);
  launch_assemble_combined(h->dc, h->d_Cc, h->d_cvec, h->d_cvec + h->dc,
                           h->d_cvec + 2 * h->dc, h->d_scal,
                           h->shift != 0.0 ? h->d_cgram : nullptr, h->shift, h->d_Sc, h->d_Hc, h->st);
  return BLM_OK;
}

bool combined_is_dense(const blm_handle* h) { return h->dc + 1 <= kDenseCombinedMax; }

// The combined eigen-solve alone (a batch launches the dense ones of all its problems at once).
blm_status combined_eig(blm_handle* h) {
  cudaStream_t st = h->st;
  Prof pr(h, PC_EIG_COMBINED);
  if (combined_is_dense(h)) {
    launch_eig(h->d_ceigp, 1, 512, st, &h->cdim, h->d_cteamctl);
  } else {
    BLM_CU(h, launch_davidson(h->d_ceigp, kDavidsonTol, kDavidsonIter, h->d_ceigw,
                              (int)(h->dc + 1), st));
    // a Davidson run that did not converge (clustered or ill-conditioned combined problems
    // from few samples) falls back to the dense solver on the same matrices
    launch_eig(h->d_ceigp + 1, 1, 512, st, &h->cdim, h->d_cteamctl);
  }
  return BLM_OK;
}

blm_status combined_post(blm_handle* h, double* dmu) {
  cudaStream_t st = h->st;
  {
    Prof pr(h, PC_UPDATE, 2);
    launch_update(h->nb, h->d_pbB, h->dc, h->d_cev, h->d_shift, h->d_vec, h->d_scal,
                  h->d_scal + 3, h->d_dmu, h->d_status + h->nb + 1, st);
  }
  BLM_CU(h, cudaMemcpyAsync(dmu, h->d_dmu, 8 * h->n, cudaMemcpyDefault, st));
  BLM_CU(h, cudaGetLastError());
  return BLM_OK;
}

blm_status enqueue_combined_solve(blm_handle* h, double* dmu) {
  blm_status s = combined_pre(h);
  if (s == BLM_OK) s = combined_eig(h);
  if (s == BLM_OK) s = combined_post(h, dmu);
  return s;
}

// Reads the status words of the whole step and the predicted energy (synchronises the stream).
blm_status combined_status(blm_handle* h, double* e_pred) {
  int32_t stat[3];
  double lam;
  BLM_CU(h, cudaMemcpyAsync(stat, h->d_status + h->nb, 12, cudaMemcpyDeviceToHost, h->st));
  BLM_CU(h, cudaMemcpyAsync(&lam, h->d_clam, 8, cudaMemcpyDeviceToHost, h->st));
  BLM_CU(h, cudaStreamSynchronize(h->st));
  BLM_CU(h, cudaGetLastError());
  if (stat[2] != 0) return fail(h, BLM_ERR_TIMEOUT, "tensor-core sweep: a bounded wait ran out");
  if (stat[0] != ST_OK) return fail(h, BLM_ERR_NUMERIC, std::string("combined: ") + status_text(stat[0]));
  if (stat[1] != ST_OK) return fail(h, BLM_ERR_NUMERIC, std::string("update: ") + status_text(stat[1]));
  *e_pred = lam;
  return BLM_OK;
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
  for (auto& it : a.items) *it.first = (char*)h->base + it.second;
  blm_status s = BLM_OK;
  // history directions
  if (h->n_old > 0) {
    const bool dev = is_device_ptr(p->old_dirs);
    e = cudaMemcpy(h->d_D, p->old_dirs, 8 * h->n_old * h->n,
                   dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
    if (e != cudaSuccess) s = cuda_fail(h, e, "copy old_dirs");
    if (s == BLM_OK && h->d_D32) launch_to_f32(h->d_D, h->d_D32, h->n_old * h->n, h->st);
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
    h->eig_dims.assign(h->nb, 0);
    h->cdim = (int32_t)(h->dc + 1);
    for (int b = 0; b < h->nb; ++b) {
      const int64_t D = h->db[b] + 1;
      h->eig_dims[b] = (int32_t)D;
      pbB[b] = ProjBlock{h->off[b], h->Mb[b], h->Kb[b], h->oc[b], 0, h->d_B + h->B_off[b], h->Mb[b],
                         h->d_B32 + h->B_off[b]};
      pbD[b] = ProjBlock{h->off[b], h->Mb[b], h->n_old, b * h->n_old, 0,
                         h->d_D ? h->d_D + h->off[b] : nullptr, h->n,
                         h->d_D32 ? h->d_D32 + h->off[b] : nullptr};
      ba[b] = BlockAsm{h->off[b], h->Mb[b], h->db[b], b, 0, h->d_C + h->C_off[b],
                       h->d_S + h->SH_off[b], h->d_H + h->SH_off[b]};
      ep[b] = EigProblem{(int)D, h->Kb[b], 0, kEigLocate32, h->d_S + h->SH_off[b], h->d_H + h->SH_off[b],
                         h->d_eigw + h->eigw_off[b], h->d_lam + h->lam_off[b],
                         h->d_evec + h->vec_off[b], h->d_status + b};
      dbk[b] = DirBlock{h->Mb[b], h->Kb[b], (int)D, 0, h->d_evec + h->vec_off[b],
                        h->d_B + h->B_off[b], h->d_status + b};
    }
    std::vector<EigProblem> cp(2);
    cp[0] = EigProblem{(int)(h->dc + 1), 1, 1, kEigLocate32, h->d_Sc, h->d_Hc, h->d_ceigw, h->d_clam,
                       h->d_cev, h->d_status + h->nb, nullptr};
    cp[1] = cp[0];
    cp[1].run_if_noconv = h->d_status + h->nb;
    if (s == BLM_OK) s = upload(h, pbB, &h->d_pbB);
    if (s == BLM_OK) s = upload(h, pbD, &h->d_pbD);
    if (s == BLM_OK) s = upload(h, ba, &h->d_asm);
    if (s == BLM_OK) s = upload(h, ep, &h->d_eigp);
    if (s == BLM_OK) s = upload(h, dbk, &h->d_dirb);
    if (s == BLM_OK) s = upload(h, cp, &h->d_ceigp);
  }
  if (s == BLM_OK && h->prec != BLM_PREC_F64) {
    // tensor-core tiles of 128 rows x 256 columns.  Operand arrays of a launch: 0 Y' rows, 1
    // w Y' rows (Y' itself when unweighted), 2 w X' rows; with history directions 3 T', 4 w T',
    // 5 w (E T' + U) rows (R of them).
    //   block b (first sweep; and the combined directions as one block in the second sweep):
    //     C_b = [Y'_b (wY'_b)^T | Y'_b (wX'_b)^T], m x 2m; column tiles never straddle the
    //     Y' | X' boundary
    //   history (Eq. 10): OT = Y' [wT' | w(ET'+U)]^T (n x 2R), XT = (wX') T'^T (n x R),
    //     TT = T' [wT' | w(ET'+U)]^T (R x 2R)
    std::vector<TcTile> t1, t2;
    auto tile = [](int am, int bm, int64_t ar, int64_t br, int64_t na, int64_t nb, double* out,
                   int64_t ld, bool view_ok) {
      TcTile t{};
      t.a_map = am;
      t.b_map = bm;
      t.a_row = (int32_t)ar;
      t.b_row = (int32_t)br;
      t.nA = (int32_t)std::min<int64_t>(128, na);
      t.nB = (int32_t)std::min<int64_t>(256, nb);
      t.a_view = view_ok && br <= ar && ar + 128 <= br + 256 ? 1 : 0;
      t.out = out;
      t.out_ld = ld;
      return t;
    };
    auto add_block = [&](std::vector<TcTile>& v, int64_t lo, int64_t m, double* out) {
      for (int64_t r0 = 0; r0 < m; r0 += 128) {
        for (int64_t c0 = 0; c0 < m; c0 += 256)
          v.push_back(tile(0, 1, lo + r0, lo + c0, m - r0, m - c0, out + r0 * 2 * m + c0, 2 * m, true));
        for (int64_t c0 = 0; c0 < m; c0 += 256)
          v.push_back(tile(0, 2, lo + r0, lo + c0, m - r0, m - c0, out + r0 * 2 * m + m + c0, 2 * m,
                           false));
      }
    };
    for (int b = 0; b < h->nb; ++b) add_block(t1, h->off[b], h->Mb[b], h->d_C + h->C_off[b]);
    // packed band tiles: 128-row bands of the parameter range, the columns of every block the
    // band touches, each product kept only where its row and column share a block (blocks far
    // smaller than a tile waste less of it this way)
    std::vector<TcTile> tp;
    std::vector<int32_t> blk_of(h->n);
    for (int b = 0; b < h->nb; ++b)
      for (int64_t x = h->off[b]; x < h->off[b + 1]; ++x) blk_of[x] = b;
    for (int64_t r0 = 0; r0 < h->n; r0 += 128) {
      const int64_t r1 = std::min<int64_t>(r0 + 128, h->n);
      const int64_t c_lo = h->off[blk_of[r0]], c_hi = h->off[blk_of[r1 - 1] + 1];
      for (int half = 1; half <= 2; ++half)
        for (int64_t c0 = c_lo; c0 < c_hi; c0 += 256) {
          TcTile t = tile(0, half, r0, c0, r1 - r0, c_hi - c0, nullptr, 0, half == 1);
          t.packed = 1;
          tp.push_back(t);
        }
    }
    std::vector<TcTile> hist;
    if (h->n_old > 0) {
      const int64_t n = h->n, R = h->R;
      for (int64_t i0 = 0; i0 < n; i0 += 128)
        for (int64_t j0 = 0; j0 < R; j0 += 256) {
          hist.push_back(tile(0, 4, i0, j0, n - i0, R - j0, h->d_OT + i0 * 2 * R + j0, 2 * R, false));
          hist.push_back(tile(0, 5, i0, j0, n - i0, R - j0, h->d_OT + i0 * 2 * R + R + j0, 2 * R, false));
          hist.push_back(tile(2, 3, i0, j0, n - i0, R - j0, h->d_XT + i0 * R + j0, R, false));
        }
      for (int64_t i0 = 0; i0 < R; i0 += 128)
        for (int64_t j0 = 0; j0 < R; j0 += 256) {
          // A = T' (array 3) is a view of B = w T' (array 4) when unweighted
          hist.push_back(tile(3, 4, i0, j0, R - i0, R - j0, h->d_TT + i0 * 2 * R + j0, 2 * R, true));
          hist.push_back(tile(3, 5, i0, j0, R - i0, R - j0, h->d_TT + i0 * 2 * R + R + j0, 2 * R,
                              false));
        }
    }
    t1.insert(t1.end(), hist.begin(), hist.end());
    tp.insert(tp.end(), hist.begin(), hist.end());
    add_block(t2, 0, h->dc, h->d_Cc);
    // the combined overlap is symmetric and assembled from its upper triangle: overlap tiles
    // (array 1) wholly below the diagonal (last column < first row) are not computed
    t2.erase(std::remove_if(t2.begin(), t2.end(),
                            [](const TcTile& t) { return t.b_map == 1 && t.b_row + 256 <= t.a_row; }),
             t2.end());
    h->ntc1_layout[0] = (int)t1.size();
    h->ntc1_layout[1] = (int)tp.size();
    h->ntc2 = (int)t2.size();
    s = upload(h, t1, &h->d_tc1_layout[0]);
    if (s == BLM_OK) s = upload(h, tp, &h->d_tc1_layout[1]);
    if (s == BLM_OK) s = upload(h, t2, &h->d_tc2);
    h->d_tc1 = h->d_tc1_layout[0];
    h->ntc1 = h->ntc1_layout[0];
    std::vector<int64_t> blo(h->off.begin(), h->off.end() - 1);
    std::vector<double*> bC(h->nb);
    for (int b = 0; b < h->nb; ++b) bC[b] = h->d_C + h->C_off[b];
    if (s == BLM_OK) s = upload(h, blk_of, &h->d_blk_of);
    if (s == BLM_OK) s = upload(h, blo, &h->d_blk_lo);
    if (s == BLM_OK) s = upload(h, h->Mb, &h->d_blk_m);
    if (s == BLM_OK) s = upload(h, bC, &h->d_blk_C);
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
  blm_status s = enqueue_block_solve(h);
  if (s != BLM_OK) return s;
  s = block_status(h);
  if (s != BLM_OK) return s;
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
  blm_status s = enqueue_combined_solve(h, dmu);
  if (s != BLM_OK) return s;
  s = combined_status(h, e_pred);
  if (s != BLM_OK) return s;
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
                  h->d_pbB, h->d_pbD, h->d_asm, h->d_eigp, h->d_ceigp, h->d_dirb,
                  h->d_tc1_layout[0], h->d_tc1_layout[1], h->d_tc2, h->d_blk_of, h->d_blk_lo,
                  h->d_blk_m, h->d_blk_C};
  for (void* p : tabs)
    if (p) cudaFree(p);
  for (int b = 0; b < 2; ++b) {
    for (int k = 0; k < 4; ++k)
      if (h->d_stage[b][k]) cudaFree(h->d_stage[b][k]);
    if (h->ev_copy[b]) cudaEventDestroy(h->ev_copy[b]);
    if (h->ev_done[b]) cudaEventDestroy(h->ev_done[b]);
  }
  if (h->copy_st) cudaStreamDestroy(h->copy_st);
  if (h->hc_pool) cudaFree(h->hc_pool);
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  if (h->graph_st) cudaStreamDestroy(h->graph_st);
  for (auto& pe : h->prof_ev) {
    cudaEventDestroy(pe.second.first);
    cudaEventDestroy(pe.second.second);
  }
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  delete h;
  return BLM_OK;
}

const char* blm_last_error(const blm_handle* h) { return h ? h->err.c_str() : "NULL handle"; }

blm_status blm_graph_capture(blm_handle* h, const void* O, const void* dEL, const void* EL,
                             const void* w, int64_t n_samples, int64_t chunk, int64_t ld,
                             double* dmu) {
  if (!h) return BLM_ERR_ARG;
  if (!O || !dEL || !EL || !dmu || n_samples <= 0 || chunk <= 0 || ld < h->n)
    return fail(h, BLM_ERR_ARG, "blm_graph_capture: bad arguments");
  if (!is_device_ptr(O) || !is_device_ptr(dEL) || !is_device_ptr(EL) || !is_device_ptr(w) ||
      !is_device_ptr(dmu))
    return fail(h, BLM_ERR_ARG, "blm_graph_capture: sample arrays and dmu must be device memory");
  if (h->graph_exec) {
    cudaGraphExecDestroy(h->graph_exec);
    h->graph_exec = nullptr;
  }
  if (!h->graph_st) BLM_CU(h, cudaStreamCreateWithFlags(&h->graph_st, cudaStreamNonBlocking));
  // work queued on the handle's stream before the capture must not overlap the captured step's
  // first launches, which the caller may replay at once
  BLM_CU(h, cudaStreamSynchronize(h->st));
  cudaStream_t user = h->st;
  const bool prof = h->prof;
  h->st = h->graph_st;
  h->prof = false;
  cudaGraph_t graph = nullptr;
  blm_status s = BLM_OK;
  cudaError_t e = cudaStreamBeginCapture(h->graph_st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    s = cuda_fail(h, e, "cudaStreamBeginCapture");
  } else {
    const bool f32 = h->in_type == BLM_IN_F32;
    s = zero_sums(h);
    for (int64_t s0 = 0; s == BLM_OK && s0 < n_samples; s0 += chunk) {
      const int64_t c = std::min(chunk, n_samples - s0);
      s = f32 ? accumulate_dev<float>(h, (const float*)O + s0 * ld, (const float*)dEL + s0 * ld,
                                      (const float*)EL + s0, w ? (const float*)w + s0 : nullptr, c, ld)
              : accumulate_dev<double>(h, (const double*)O + s0 * ld, (const double*)dEL + s0 * ld,
                                       (const double*)EL + s0, w ? (const double*)w + s0 : nullptr,
                                       c, ld);
    }
    if (s == BLM_OK) s = enqueue_block_solve(h);
    for (int64_t s0 = 0; s == BLM_OK && s0 < n_samples; s0 += chunk) {
      const int64_t c = std::min(chunk, n_samples - s0);
      s = f32 ? project_dev<float>(h, (const float*)O + s0 * ld, (const float*)dEL + s0 * ld,
                                   (const float*)EL + s0, w ? (const float*)w + s0 : nullptr, c, ld)
              : project_dev<double>(h, (const double*)O + s0 * ld, (const double*)dEL + s0 * ld,
                                    (const double*)EL + s0, w ? (const double*)w + s0 : nullptr,
                                    c, ld);
    }
    if (s == BLM_OK) s = enqueue_combined_solve(h, dmu);
    e = cudaStreamEndCapture(h->graph_st, &graph);
    if (s == BLM_OK && e != cudaSuccess) s = cuda_fail(h, e, "cudaStreamEndCapture");
  }
  h->st = user;
  h->prof = prof;
  h->state = ST_CREATED;
  if (s == BLM_OK) {
    e = cudaGraphInstantiate(&h->graph_exec, graph, 0);
    if (e != cudaSuccess) {
      h->graph_exec = nullptr;
      s = cuda_fail(h, e, "cudaGraphInstantiate");
    }
  }
  if (graph) cudaGraphDestroy(graph);
  cudaGetLastError();
  return s;
}

blm_status blm_batch_destroy(blm_batch* b) {
  if (!b) return BLM_OK;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (blm_handle* h : b->hs) blm_destroy(h);
  for (cudaEvent_t e : b->ev)
    if (e) cudaEventDestroy(e);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->cap_st) cudaStreamDestroy(b->cap_st);
  if (b->d_blocks) cudaFree(b->d_blocks);
  if (b->d_comb) cudaFree(b->d_comb);
  if (b->d_teamctl) cudaFree(b->d_teamctl);
  delete b;
  return BLM_OK;
}

blm_status blm_batch_create(const blm_problem* problems, int32_t count, void* stream,
                            blm_batch** out) {
  if (!out) return BLM_ERR_ARG;
  *out = nullptr;
  if (!problems || count <= 0) return BLM_ERR_ARG;
  blm_batch* b = new blm_batch();
  b->st = (cudaStream_t)stream;
  std::vector<EigProblem> blocks, comb;
  blm_status s = BLM_OK;
  for (int i = 0; i < count && s == BLM_OK; ++i) {
    blm_handle* h = nullptr;
    s = blm_create(&problems[i], stream, &h);
    if (s != BLM_OK) {
      fprintf(stderr, "blm_batch_create: problem %d rejected\n", i);
      break;
    }
    b->hs.push_back(h);
    std::vector<EigProblem> ep(h->nb), cp(2);
    if (cudaMemcpy(ep.data(), h->d_eigp, sizeof(EigProblem) * h->nb, cudaMemcpyDeviceToHost) !=
            cudaSuccess ||
        cudaMemcpy(cp.data(), h->d_ceigp, sizeof(EigProblem) * 2, cudaMemcpyDeviceToHost) !=
            cudaSuccess) {
      s = BLM_ERR_CUDA;
      break;
    }
    blocks.insert(blocks.end(), ep.begin(), ep.end());
    b->blk_dims.insert(b->blk_dims.end(), h->eig_dims.begin(), h->eig_dims.end());
    if (combined_is_dense(h)) {
      comb.push_back(cp[0]);
      b->comb_dims.push_back(h->cdim);
    }
  }
  if (s == BLM_OK) {
    b->nblocks_all = (int)blocks.size();
    b->ncomb_dense = (int)comb.size();
    b->ev.assign(count, nullptr);
    bool ok = cudaMalloc((void**)&b->d_blocks, sizeof(EigProblem) * blocks.size()) == cudaSuccess &&
              cudaMemcpy(b->d_blocks, blocks.data(), sizeof(EigProblem) * blocks.size(),
                         cudaMemcpyHostToDevice) == cudaSuccess;
    if (ok)
      ok = cudaMalloc(&b->d_teamctl, eig_team_ctl_bytes((int)blocks.size()) +
                                         eig_team_ctl_bytes((int)comb.size())) == cudaSuccess;
    if (ok && !comb.empty())
      ok = cudaMalloc((void**)&b->d_comb, sizeof(EigProblem) * comb.size()) == cudaSuccess &&
           cudaMemcpy(b->d_comb, comb.data(), sizeof(EigProblem) * comb.size(),
                      cudaMemcpyHostToDevice) == cudaSuccess;
    for (int i = 0; ok && i < count; ++i)
      ok = cudaEventCreateWithFlags(&b->ev[i], cudaEventDisableTiming) == cudaSuccess &&
           (b->hs[i]->graph_st ||
            cudaStreamCreateWithFlags(&b->hs[i]->graph_st, cudaStreamNonBlocking) == cudaSuccess);
    ok = ok && cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
         cudaStreamCreateWithFlags(&b->cap_st, cudaStreamNonBlocking) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      s = BLM_ERR_NOMEM;
    }
  }
  if (s != BLM_OK) {
    blm_batch_destroy(b);
    return s;
  }
  *out = b;
  return BLM_OK;
}

blm_handle* blm_batch_handle(blm_batch* b, int32_t i) {
  if (!b || i < 0 || i >= (int32_t)b->hs.size()) return nullptr;
  return b->hs[i];
}

const char* blm_batch_last_error(const blm_batch* b) { return b ? b->err.c_str() : "NULL batch"; }

blm_status blm_batch_capture(blm_batch* b, const void* const* O, const void* const* dEL,
                             const void* const* EL, const void* const* w,
                             const int64_t* n_samples, const int64_t* ld, int64_t chunk,
                             double* const* dmu) {
  if (!b || !O || !dEL || !EL || !n_samples || !ld || !dmu || chunk <= 0) return BLM_ERR_ARG;
  const int count = (int)b->hs.size();
  for (int i = 0; i < count; ++i) {
    blm_handle* h = b->hs[i];
    const void* wi = w ? w[i] : nullptr;
    if (!O[i] || !dEL[i] || !EL[i] || !dmu[i] || n_samples[i] <= 0 || ld[i] < h->n ||
        !is_device_ptr(O[i]) || !is_device_ptr(dEL[i]) || !is_device_ptr(EL[i]) ||
        !is_device_ptr(wi) || !is_device_ptr(dmu[i])) {
      b->err = "blm_batch_capture: bad arguments or host memory for problem " + std::to_string(i);
      return BLM_ERR_ARG;
    }
  }
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  if (cudaStreamSynchronize(b->st) != cudaSuccess) return BLM_ERR_CUDA;
  std::vector<cudaStream_t> user(count);
  std::vector<bool> prof(count);
  for (int i = 0; i < count; ++i) {
    user[i] = b->hs[i]->st;
    prof[i] = b->hs[i]->prof;
    b->hs[i]->prof = false;
  }
  cudaGraph_t graph = nullptr;
  blm_status s = BLM_OK;
  cudaError_t e = cudaStreamBeginCapture(b->cap_st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    b->err = std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e);
    s = BLM_ERR_CUDA;
  }
  // one branch per problem between joins; the eigen-solves of all problems in shared launches
  auto fork = [&]() {
    cudaEventRecord(b->ev_fork, b->cap_st);
    for (int i = 0; i < count; ++i) {
      b->hs[i]->st = b->hs[i]->graph_st;
      cudaStreamWaitEvent(b->hs[i]->graph_st, b->ev_fork, 0);
    }
  };
  auto join = [&]() {
    for (int i = 0; i < count; ++i) {
      cudaEventRecord(b->ev[i], b->hs[i]->graph_st);
      cudaStreamWaitEvent(b->cap_st, b->ev[i], 0);
    }
  };
  auto sweep_all = [&](int pass, int i) -> blm_status {
    blm_handle* h = b->hs[i];
    const bool f32 = h->in_type == BLM_IN_F32;
    const int64_t ns = n_samples[i], l = ld[i];
    const void* wi = w ? w[i] : nullptr;
    blm_status r = BLM_OK;
    for (int64_t s0 = 0; r == BLM_OK && s0 < ns; s0 += chunk) {
      const int64_t c = std::min(chunk, ns - s0);
      if (f32) {
        const float* o = (const float*)O[i] + s0 * l;
        const float* g = (const float*)dEL[i] + s0 * l;
        const float* en = (const float*)EL[i] + s0;
        const float* ww = wi ? (const float*)wi + s0 : nullptr;
        r = pass == 1 ? accumulate_dev<float>(h, o, g, en, ww, c, l)
                      : project_dev<float>(h, o, g, en, ww, c, l);
      } else {
        const double* o = (const double*)O[i] + s0 * l;
        const double* g = (const double*)dEL[i] + s0 * l;
        const double* en = (const double*)EL[i] + s0;
        const double* ww = wi ? (const double*)wi + s0 : nullptr;
        r = pass == 1 ? accumulate_dev<double>(h, o, g, en, ww, c, l)
                      : project_dev<double>(h, o, g, en, ww, c, l);
      }
    }
    return r;
  };
  if (s == BLM_OK) {
    fork();
    for (int i = 0; s == BLM_OK && i < count; ++i) {
      s = zero_sums(b->hs[i]);
      if (s == BLM_OK) s = sweep_all(1, i);
      if (s == BLM_OK) s = block_solve_pre(b->hs[i]);
    }
    join();
    if (s == BLM_OK)
      launch_eig(b->d_blocks, b->nblocks_all, 512, b->cap_st, b->blk_dims.data(), b->d_teamctl);
    fork();
    for (int i = 0; s == BLM_OK && i < count; ++i) {
      s = block_solve_post(b->hs[i]);
      if (s == BLM_OK) s = sweep_all(2, i);
      if (s == BLM_OK) s = combined_pre(b->hs[i]);
    }
    join();
    if (s == BLM_OK && b->ncomb_dense > 0)
      launch_eig(b->d_comb, b->ncomb_dense, 512, b->cap_st, b->comb_dims.data(),
                 static_cast<char*>(b->d_teamctl) + eig_team_ctl_bytes(b->nblocks_all));
    // combined problems above the dense limit: Davidson (a cooperative grid over every SM),
    // one at a time on the origin stream while no branch runs
    for (int i = 0; s == BLM_OK && i < count; ++i)
      if (!combined_is_dense(b->hs[i])) {
        b->hs[i]->st = b->cap_st;
        s = combined_eig(b->hs[i]);
      }
    fork();
    for (int i = 0; s == BLM_OK && i < count; ++i) s = combined_post(b->hs[i], dmu[i]);
    join();
    e = cudaStreamEndCapture(b->cap_st, &graph);
    if (s == BLM_OK && e != cudaSuccess) {
      b->err = std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e);
      s = BLM_ERR_CUDA;
    }
  }
  for (int i = 0; i < count; ++i) {
    if (s != BLM_OK && b->err.empty()) b->err = b->hs[i]->err;
    b->hs[i]->st = user[i];
    b->hs[i]->prof = prof[i];
    b->hs[i]->state = ST_CREATED;
  }
  if (s == BLM_OK) {
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    if (e != cudaSuccess) {
      b->exec = nullptr;
      b->err = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e);
      s = BLM_ERR_CUDA;
    }
  }
  if (graph) cudaGraphDestroy(graph);
  cudaGetLastError();
  return s;
}

blm_status blm_batch_launch(blm_batch* b) {
  if (!b) return BLM_ERR_ARG;
  if (!b->exec) {
    b->err = "blm_batch_launch: no captured step";
    return BLM_ERR_STATE;
  }
  cudaError_t e = cudaGraphLaunch(b->exec, b->st);
  if (e != cudaSuccess) {
    b->err = std::string("cudaGraphLaunch: ") + cudaGetErrorString(e);
    return BLM_ERR_CUDA;
  }
  return BLM_OK;
}

blm_status blm_batch_result(blm_batch* b, double* e_pred, int32_t* status) {
  if (!b || !e_pred) return BLM_ERR_ARG;
  if (!b->exec) {
    b->err = "blm_batch_result: no captured step";
    return BLM_ERR_STATE;
  }
  blm_status first = BLM_OK;
  for (size_t i = 0; i < b->hs.size(); ++i) {
    blm_handle* h = b->hs[i];
    blm_status s = block_status(h);
    if (s == BLM_OK) s = combined_status(h, &e_pred[i]);
    if (s == BLM_OK) h->state = ST_DONE;
    else e_pred[i] = NAN;
    if (status) status[i] = s;
    if (s != BLM_OK && first == BLM_OK) {
      first = s;
      b->err = "problem " + std::to_string(i) + ": " + h->err;
    }
  }
  return first;
}

blm_status blm_set_tiles(blm_handle* h, int32_t choice) {
  if (!h) return BLM_ERR_ARG;
  if (choice < 0 || choice > 3) return fail(h, BLM_ERR_ARG, "blm_set_tiles: choice outside 0..3");
  if (h->prec == BLM_PREC_F64) return BLM_OK;
  BLM_CU(h, cudaStreamSynchronize(h->st));
  h->layout = choice >> 1;
  h->d_tc1 = h->d_tc1_layout[h->layout];
  h->ntc1 = h->ntc1_layout[h->layout];
  h->tc_range_max = (choice & 1) ? 4096 : 16384;
  return BLM_OK;
}

blm_status blm_autotune(blm_handle* h, const void* O, const void* dEL, const void* EL,
                        const void* w, int64_t n_samples, int64_t ld, int32_t* choice) {
  if (!h) return BLM_ERR_ARG;
  if (choice) *choice = 0;
  if (h->prec == BLM_PREC_F64) return BLM_OK;      // nothing to choose on the FP64 path
  if (!O || !dEL || !EL || n_samples <= 0 || ld < h->n || h->in_type != BLM_IN_F32 ||
      !is_device_ptr(O) || !is_device_ptr(dEL) || !is_device_ptr(EL) || !is_device_ptr(w))
    return fail(h, BLM_ERR_ARG, "blm_autotune: device FP32 sample arrays needed");
  const int64_t ns = std::min(n_samples, h->sub_chunk);
  const bool prof = h->prof;
  h->prof = false;
  cudaEvent_t e0, e1;
  BLM_CU(h, cudaEventCreate(&e0));
  BLM_CU(h, cudaEventCreate(&e1));
  // candidates: tile layout (per block, packed bands) x longest work unit (16384, 4096 samples)
  const int64_t ranges[2] = {16384, 4096};
  float best = 0.0f;
  int best_c = 0;
  blm_status s = BLM_OK;
  for (int c = 0; c < 4 && s == BLM_OK; ++c) {
    h->layout = c >> 1;
    h->d_tc1 = h->d_tc1_layout[h->layout];
    h->ntc1 = h->ntc1_layout[h->layout];
    h->tc_range_max = ranges[c & 1];
    float t_min = 0.0f;
    for (int rep = 0; rep < 3 && s == BLM_OK; ++rep) {
      s = zero_sums(h);
      if (s != BLM_OK) break;
      BLM_CU(h, cudaEventRecord(e0, h->st));
      s = accumulate_dev<float>(h, (const float*)O, (const float*)dEL, (const float*)EL,
                                (const float*)w, ns, ld);
      BLM_CU(h, cudaEventRecord(e1, h->st));
      BLM_CU(h, cudaEventSynchronize(e1));
      float ms = 0.0f;
      BLM_CU(h, cudaEventElapsedTime(&ms, e0, e1));
      if (rep > 0 && (rep == 1 || ms < t_min)) t_min = ms;   // the first run warms up
    }
    if (s == BLM_OK && (c == 0 || t_min < best)) {
      best = t_min;
      best_c = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->layout = best_c >> 1;
  h->d_tc1 = h->d_tc1_layout[h->layout];
  h->ntc1 = h->ntc1_layout[h->layout];
  h->tc_range_max = ranges[best_c & 1];
  h->prof = prof;
  if (s == BLM_OK) s = zero_sums(h);
  if (s == BLM_OK) {
    int32_t st[1];
    BLM_CU(h, cudaMemcpyAsync(st, h->d_status + h->nb + 2, 4, cudaMemcpyDeviceToHost, h->st));
    BLM_CU(h, cudaStreamSynchronize(h->st));
  }
  if (choice) *choice = best_c;
  return s;
}

blm_status blm_graph_launch(blm_handle* h) {
  if (!h) return BLM_ERR_ARG;
  if (!h->graph_exec) return fail(h, BLM_ERR_STATE, "blm_graph_launch: no captured step");
  BLM_CU(h, cudaGraphLaunch(h->graph_exec, h->st));
  return BLM_OK;
}

blm_status blm_graph_result(blm_handle* h, double* e_pred) {
  if (!h || !e_pred) return BLM_ERR_ARG;
  if (!h->graph_exec) return fail(h, BLM_ERR_STATE, "blm_graph_result: no captured step");
  blm_status s = block_status(h);
  if (s != BLM_OK) return s;
  s = combined_status(h, e_pred);
  if (s != BLM_OK) return s;
  h->state = ST_DONE;
  return BLM_OK;
}

blm_status blm_set_host_cache(blm_handle* h, size_t bytes) {
  if (!h) return BLM_ERR_ARG;
  BLM_CU(h, cudaStreamSynchronize(h->st));
  if (h->hc_pool) cudaFree(h->hc_pool);
  h->hc_pool = nullptr;
  h->hc_capacity = h->hc_used = 0;
  h->hc_pieces.clear();
  if (bytes == 0) return BLM_OK;
  if (cudaMalloc((void**)&h->hc_pool, bytes) != cudaSuccess) {
    cudaGetLastError();
    h->hc_pool = nullptr;
    return fail(h, BLM_ERR_NOMEM, "blm_set_host_cache: device allocation failed");
  }
  h->hc_capacity = bytes;
  return BLM_OK;
}

blm_status blm_set_wait_limit(blm_handle* h, uint32_t polls) {
  if (!h) return BLM_ERR_ARG;
  h->wait_limit = polls;
  return BLM_OK;
}

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
