// Internal interface between the host orchestration (api.cu) and the kernel
// translation units.  Nothing here is part of the public C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "common.cuh"

namespace figaro {

constexpr int kMaxWidth = 128;          // n1 + n2 limit of the one-CTA dense n x n kernels
constexpr int kMaxWideWidth = 512;      // n1 + n2 limit of the wide (multi-CTA) path
constexpr int kMaxTableWidth = 256;     // per-table width limit of the wide path
constexpr int kSortThreads = 512;
constexpr int kSortItems = 13;  // 6,656-key tiles: 2 x 151 tiles for 1e6-row tables fill 152 SMs twice
constexpr int kSortTile = kSortThreads * kSortItems;  // keys per radix tile
constexpr int kRadixBits = 8;
constexpr int kRadixBins = 1 << kRadixBits;
constexpr int kMaxPasses = 4;
constexpr int kGramThreads = 256;
constexpr int kGramTileRows = 64;
constexpr int kReduceWarps = 16;  // warps of a Gram-reduce CTA

constexpr int kMaxJacobiBlocks = 160;  // column blocks of the wide Jacobi (n <= 512 in blocks of >= 4)

// Device-side header at the start of every workspace.
struct alignas(256) DevHeader {
  int32_t status;            // figaro status bits (common.cuh)
  int32_t report_rank;       // a dropped column k < report_rank makes the status FIGARO_ERR_RANK_DEFICIENT
  uint32_t ticket[8];        // persistent-grid work tickets
  uint32_t kmin[2];          // ordered-key range per table (A = 0, B = 1)
  uint32_t kmax[2];
  int64_t num_runs[2];
  int64_t num_groups;
  int64_t reduced_rows;      // sum over matched keys of (m1g + m2g - 1)
  int32_t jacobi_sweeps;
  int32_t dep_cols;          // columns the last factorisation marked dependent (zero rows of R)
  uint32_t bar_count;        // grid barrier of the cooperative dense kernels (wide path)
  uint32_t bar_gen;
  uint32_t sweep_any[3];     // per-sweep "a pair was rotated" flags of the wide Jacobi
  uint32_t pad2;
  uint32_t blk_ver[kMaxJacobiBlocks];  // wide Jacobi: rounds completed on each column block
};

// Per-table buffers of the grouping and head/tail steps.
struct TableWork {
  // input (device; staged copy when the caller passed host memory)
  const void* x = nullptr;
  const int32_t* key = nullptr;
  int64_t m = 0;
  int64_t ld = 0;
  int n = 0;
  int in_f64 = 0;            // input element type: 1 = double, 0 = float
  // grouping
  uint32_t* kb[2] = {nullptr, nullptr};
  int32_t* vb[2] = {nullptr, nullptr};
  uint32_t* hist = nullptr;          // kMaxPasses x kRadixBins global digit counts
  uint64_t* sort_status = nullptr;   // per-tile digit counts and offsets: kMaxPasses x tiles x kRadixBins words
  uint64_t* run_status = nullptr;    // per-tile run counts: tiles words
  int tiles = 0;
  int32_t* perm = nullptr;
  int32_t* sorted_key = nullptr;
  int32_t* seg = nullptr;       // run index of each sorted row
  int32_t* run_key = nullptr;
  int32_t* run_off = nullptr;   // m + 1
  int32_t* other = nullptr;     // partner run size (0 = unmatched)
  int32_t* hdslot = nullptr;    // head row of the run's key group
  int32_t* run_info = nullptr;  // per run: {first row, end row, partner run size, head slot}
  int32_t* lut = nullptr;       // key lookup table: run index at (ordered key - smallest key of both tables)
  // head/tail
  void* tail = nullptr;         // m x n slots, compute type
  int chunk_rows = 0;           // chunk spacing L of the head/tail step
  int chunks = 0;               // ceil(m / L)
  int32_t* cbeg = nullptr;      // chunks + 1 first rows
  uint32_t* cflag = nullptr;    // chunks flags
  double* piece = nullptr;      // chunks x n long-run piece sums
  double* carry = nullptr;      // chunks x n carries
};

// Everything one instance needs, resolved from the workspace.
struct Plan {
  TableWork t[2];
  int n1 = 0, n2 = 0, n = 0;
  int mixed = 1;                // 1 = mixed path (FP32 compute), 0 = plain FP64
  int gram_engine = 1;
  int max_sweeps = 40;
  int64_t spin_limit = 0;
  double rank_tol = 0.0;
  int withhold = 0;             // test-only fault injection (see FIGARO_FLAG_TEST_WITHHOLD)
  int report_rank = 0;          // leading columns whose drop raises FIGARO_ERR_RANK_DEFICIENT (0: none)
  int shifted = 0;              // shifted CholeskyQR3: shift G1, then a third Gram pass
  int presorted = 0;            // the tables are in key order: no radix sort (identity permutation)
  int sigma_dqds = 0;           // singular values by bidiagonalisation and dqds instead of Jacobi
  // pass 1 of the tail blocks inside the head/tail stream (ht_plan_gram1):
  // the stream's CTAs per table, and per table the number of float-float
  // Gram partials of its tails those CTAs write (0: the Gram pass reads the tails)
  int ht_grid[2] = {0, 0};
  int ht_gram[2] = {0, 0};
  int ht_split = 0;  // the head/tail step runs per table (host-staged tables), each launch on the whole GPU
  int64_t lut_size = 0;         // entries of each table's key lookup table
  DevHeader* hdr = nullptr;
  void* head = nullptr;         // m1 x n slots, compute type
  // Gram partials: [grid x slices x k x k] doubles per block
  double* gpart[3] = {nullptr, nullptr, nullptr};
  int ggrid[3] = {0, 0, 0};
  int gslices[3] = {0, 0, 0};
  // small dense n x n (doubles unless noted)
  double* G1 = nullptr;
  double* G2 = nullptr;
  double* R1 = nullptr;
  double* W = nullptr;
  float* Wf = nullptr;
  double* R = nullptr;
  double* sigma = nullptr;
  int32_t* active = nullptr;
  int num_sms = 148;
  // wide path (n1 + n2 > kMaxWidth): Q = X W per Gram block, 64 x 64 tile
  // partials, and n x n work arrays of the multi-CTA dense steps
  int wide = 0;
  void* wq[3] = {nullptr, nullptr, nullptr};  // head (m1 x n), A tails (m1 x n), B tails (m2 x n2)
  double* wpart = nullptr;                    // wide Gram partials (64 x 64 or 128 x 128 doubles per job)
  float* wt = nullptr;                        // mixed wide path: W^T (n x n) and its TF32 lo parts
  float* wtlo = nullptr;
  void* Aw = nullptr;                         // n x n compute type (in-place Cholesky)
  void* Tw = nullptr;                         // n x n compute type (inverse)
  double* Xw = nullptr;                       // n x n FP64 (refined R1)
  void* Uw = nullptr;                         // Jacobi columns: (n + 32) x n compute type
  void* Vw = nullptr;
  void* yw = nullptr;                         // n pivots 1 / sqrt(d)
  void* d0w = nullptr;                        // n diagonal of the factored Gram
  double* sigw = nullptr;                     // 2n: unsorted singular values, FP32-sweep column norms
  // batched calls: Gram partials written per (pass, block) and their format
  // (0 FP64 upper triangle, 1 FP64 P with G = (P + P^T) / 2 from the general
  // tensor-core engine, 2 float-float pairs from the packed engine, 3 FP64
  // 128 x 128 tiles from the tile Gram)
  int gcount[2][3] = {{0, 0, 0}, {0, 0, 0}};
  int gsym[2][3] = {{0, 0, 0}, {0, 0, 0}};
  int64_t gcap[3] = {0, 0, 0};  // doubles of gpart[b]
};

// Batched execution (figaro_batch_join): every instance's plan sits in device
// memory, and each batched launch gets a job list that maps its CTAs to
// (instance, CTA within the job): job j owns CTAs [first[j], first[j+1]).
struct BatchJobs {
  const int32_t* first;  // njobs + 1
  const int32_t* inst;   // njobs: instance index
  const int32_t* aux;    // njobs: job detail (table, Gram block, ...)
  int njobs;
  int ctas;              // first[njobs]
};

// Per-instance outputs of a batch.
struct BatchOut {
  double* R;             // n x n, leading dimension n (device), or null
  double* sigma;         // n (device), or null
};

struct BatchDev {
  const Plan* plans;     // count plans (device)
  const BatchOut* out;   // count outputs (device)
  int count;
};

// The workspace header that holds a status word (the header's first member).
__device__ __forceinline__ DevHeader* header_of(int32_t* status) { return reinterpret_cast<DevHeader*>(status); }

// A factorisation marked column k dependent although its norm is not zero:
// recorded as FIGARO_ERR_RANK_DEFICIENT when the call reports column k.
__device__ __forceinline__ void note_dropped(int32_t* status, int k) {
  if (k < header_of(status)->report_rank) set_status(status, kStatusRankDrop);
}

// Job j of a launch for CTA b (binary search over first[]).
__device__ __forceinline__ int batch_job(const BatchJobs& J, int b) {
  int lo = 0, hi = J.njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (J.first[mid] <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Launch with programmatic stream serialization: the kernel may be scheduled
// while the previous kernel in the stream finishes (every kernel of this
// library calls pdl_enter() first, which waits for that kernel).
template <typename... KArgs, typename... Args>
cudaError_t pdl_launch(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<Args&&>(args)...);
}

// cuTensorMapEncodeTiled from the driver (null when unavailable).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

// Look-back words the grouping step needs per table (sort passes + runs).
int64_t group_status_words(int tiles);

// Host-side count of kernel launches (figaro_kernel_launches()).
void count_launches(int n);

// Sizes the plan from shapes alone (device pointers stay null when
// ws == nullptr).  Returns the workspace bytes needed.
size_t plan_layout(Plan& p, const void* ws_base, int64_t m1, int n1, int64_t m2, int n2, int in_f64, int mixed,
                   int stage_a, int stage_b, int num_sms);

// Launchers (each returns the first CUDA error it meets).
cudaError_t launch_reset(const Plan& p, cudaStream_t s);
cudaError_t launch_grouping(const Plan& p, cudaStream_t s);
// only: the table to process (-1: both in one launch)
cudaError_t launch_ht_carry(const Plan& p, cudaStream_t s, int only = -1);
cudaError_t launch_ht_main(const Plan& p, cudaStream_t s, int only = -1);
// Decides, before launch_ht_main, which tables' pass-1 Gram partials the
// head/tail stream accumulates (mixed path, FP32 tables of 8 or 16
// columns on the 4-column consumers, automatic Gram engine).
void ht_plan_gram1(Plan& p);
cudaError_t launch_gram_pass(const Plan& p, int pass, cudaStream_t s);
cudaError_t launch_chol_first(const Plan& p, cudaStream_t s);
// Shifted CholeskyQR3 between its second and third passes: R1 = R (the
// second pass's factor), W = R^{-1} on the columns with a non-zero diagonal.
cudaError_t launch_refactor(const Plan& p, cudaStream_t s);
cudaError_t launch_chol_second(const Plan& p, double* R_out, int64_t ldr, cudaStream_t s);
cudaError_t launch_jacobi(const Plan& p, const double* R, int64_t ldr, double* sigma, cudaStream_t s);
// Singular values by bidiagonalisation and dqds (sigma.cu; n <= kMaxWidth):
// one CTA per matrix; the header's sweep counter receives the number of dqds
// transforms, or -1 when dqds stopped early.  mixed = 1: FP32 stages; 0:
// FP64 bidiagonalisation and float-float dqds (also the direct entry point).
size_t sigma_dqds_smem(int n, int mixed);
int sigma_dqds_threads();
cudaError_t launch_sigma_dqds(const Plan& p, const double* R, int64_t ldr, double* sigma, cudaStream_t s);
cudaError_t launch_sigma_dqds_many(const double* R, int64_t ldr, int64_t stride, int n, int count, double* sigma,
                                   int32_t* info, cudaStream_t s);
cudaError_t launch_lsq(const Plan& p, double* beta, double* residual, cudaStream_t s);

// Batched launchers: every instance of a batch in one launch per phase.
//   tiles: one job per (instance, table with rows), CTAs = radix tiles, aux = table
//   match: one job per instance, CTAs = ceil(max(m1, m2) / 256)
cudaError_t launch_batch_grouping(const BatchDev& b, const BatchJobs& tiles, const BatchJobs& match, cudaStream_t s);
//   head/tail: plan jobs count chunks (plan_total in all), scan jobs count
//   columns, stream[0] / stream[1] are the 4-column / scalar-path tables
//   (CTAs per table), smem[] their dynamic shared memory
void ht_batch_table(const Plan& p, int t, int* variant, int* smem, int* chunks);
cudaError_t launch_batch_ht(const BatchDev& b, const BatchJobs& plan, int plan_total, const BatchJobs& scan,
                            const BatchJobs stream[2], const int smem[2], int in_f64, int mixed, cudaStream_t s);

//   Gram (CUDA cores): by_tpt[v] = (instance, block) jobs of variant v with
//   the block's CTAs (aux = block), reduce = one job per instance
void gram_batch_block(const Plan& p, int pass, int b, int* variant, int* ctas, size_t* smem);
// gargs / rargs: device arrays of the jobs' Gram arguments ([instance][block])
// and reduce arguments ([instance]) for this pass, written by
// launch_batch_args (null: each CTA derives its own from the plan)
cudaError_t launch_batch_gram(const BatchDev& b, int pass, const BatchJobs by_tpt[4], const size_t smem[4],
                              const BatchJobs& reduce, int mixed, const void* gargs, const void* rargs,
                              cudaStream_t s);
size_t batch_gram_args_bytes();
size_t batch_reduce_args_bytes();
cudaError_t launch_batch_args(const BatchDev& b, int pass, void* gargs, void* rargs, cudaStream_t s);

//   dense n x n steps (step 1, 2, 3 = first Cholesky, second Cholesky + R,
//   Jacobi): one CTA per instance, jobs[v] the instances of variant v
void dense_batch_info(const Plan& p, int step, int* variant, size_t* smem, int* threads);
cudaError_t launch_batch_dense(const BatchDev& b, int step, const BatchJobs jobs[3], const size_t smem[3],
                               const int threads[3], int mixed, cudaStream_t s);
//   the sigma step by dqds instead of Jacobi: one CTA per instance
cudaError_t launch_batch_sigma_dqds(const BatchDev& b, const BatchJobs& J, size_t smem, int mixed, cudaStream_t s);

//   Gram (tensor cores): jobs of one engine variant, in launches of up to
//   192 jobs whose tensor maps travel as kernel arguments
struct TcJob {
  int inst, blk, ctas;
};
int gram_tc_batch_engine(const Plan& p, int pass, int b, int* variant, int64_t* tile_rows, size_t* smem);
cudaError_t launch_gram_tc_batch(const Plan* dev_plans, const Plan* host_plans, int pass, int engine, int variant,
                                 const TcJob* jobs, int njobs, size_t smem, cudaStream_t s);

// Wide path (wide.cu).
// Doubles of the wide Gram partial buffer (both engines' jobs of either pass).
int64_t wide_gram_part_doubles(int64_t m1, int n1, int64_t m2, int n2, int num_sms, int mixed);
cudaError_t launch_wide_gram_pass(const Plan& p, int pass, cudaStream_t s);

// Tensor-core Gram of wide FP32 blocks (gram_tc.cu): for each block b with
// njobs > 0, one CTA per (upper 128 x 128 tile pair, row split) writes the
// tile's sum over its split as 128 x 128 doubles at part + pbase + job * 16384
// (job = tile index * splits + split; a job's rows are [split * split_rows,
// min(rows, (split + 1) * split_rows)) with rows = min(rows, *rows_dev)).
// X is row-major FP32 (ld elements, ld and the base 16-byte aligned).
constexpr int kWideTcTile = 128;
struct WideTcBlock {
  const float* X;
  int64_t ld;
  int kout;
  int64_t rows;
  const int64_t* rows_dev;
  int tiles, splits;
  int64_t split_rows;
  int njobs;
  int64_t pbase;
  double* part = nullptr;      // table launches: the block's partials (job j at part + j x 128^2)
  int32_t* status = nullptr;   // table launches: the block's device status word
};
bool wide_tc_eligible(const float* X, int64_t ld, int kout);

// Tensor-core formation Q = X W[w0:w0+k, w0:w0+kout] of wide FP32 blocks
// (gram_tc.cu), 3 x TF32: one CTA per (128-column tile of Q, range of
// rt_per_split 128-row tiles).  WT / WTlo: W^T (n x n row-major, W upper
// triangular) and its TF32 lo parts, from launch_wide_form_prep.
struct WideFormBlock {
  const float* X;
  int64_t ldx;
  int k, kout, w0;
  int64_t rows;
  const int64_t* rows_dev;
  float* Q;  // rows x kout, leading dimension kout
  int ctiles, splits, rt_per_split, njobs;
  const float* WT = nullptr;    // table launches: W^T and its lo parts (n x n) of the block's instance
  const float* WTlo = nullptr;
  int n = 0;
  int32_t* status = nullptr;    // table launches: the block's device status word
};
cudaError_t launch_wide_form_prep(const float* W, int n, float* WT, float* WTlo, cudaStream_t s);

// Table launches of the two wide tensor-core kernels (batched calls): one
// launch covers any number of blocks, each with its own tensor maps, status
// word and partials, read from device memory (entries 128-byte aligned, the
// alignment of CUtensorMap, copied there before the launch); job0[i] = the first CTA of entry i, job0[nb] = all
// CTAs.  The W^T preparation of many instances runs the same way.
struct alignas(128) WideTcEntry {
  CUtensorMap map;
  WideTcBlock b;
};
struct alignas(128) WideFormEntry {
  CUtensorMap xmap, wmap, wlmap;
  WideFormBlock b;
};
struct WidePrepEntry {
  const float* W;
  float* WT;
  float* WTlo;
  int n;
};
bool wide_tc_encode(const WideTcBlock& b, WideTcEntry* e);      // false: not addressable by TMA
bool wide_form_encode(const WideFormBlock& b, WideFormEntry* e);
cudaError_t launch_wide_gram_tc_table(const WideTcEntry* e, const int32_t* job0, int nb, int ctas,
                                      int64_t spin_limit, cudaStream_t s);
cudaError_t launch_wide_form_tc_table(const WideFormEntry* e, const int32_t* job0, int nb, int ctas,
                                      int64_t spin_limit, cudaStream_t s);
cudaError_t launch_wide_prep_table(const WidePrepEntry* e, const int32_t* cta0, int nb, int ctas, cudaStream_t s);
// Narrow mixed plans with n in (64, 128]: the head rows (both passes) and
// the A tails (pass 2) on the tensor-core formation and tile Gram (wide.cu);
// partials of block b in the reduce's format 3.
bool narrow_tc(const Plan& p, int pass, int b);
// rows_min: the fewest rows of a split (rounded up to 1024)
int narrow_tc_splits(const Plan& p, int b, int64_t rows_min, int64_t* split_rows);
// the formation (pass 2) and tile Gram blocks of block b (splits of >= rows_min rows)
void narrow_tc_blocks(const Plan& p, int pass, int b, int64_t rows_min, WideFormBlock* fb, WideTcBlock* tb);
// single calls: blocks 0 and 1 where use[b], partial counts into count[b]
cudaError_t launch_narrow_tc(const Plan& p, int pass, const bool use[3], int count[3], cudaStream_t s);
cudaError_t launch_wide_form_tc(const WideFormBlock b[3], const float* WT, const float* WTlo, int n, int32_t* status,
                                int64_t spin_limit, cudaStream_t s);
cudaError_t launch_wide_gram_tc(const WideTcBlock b[3], double* part, int32_t* status, int64_t spin_limit,
                                cudaStream_t s);
cudaError_t launch_wide_chol_first(const Plan& p, cudaStream_t s);
cudaError_t launch_wide_refactor(const Plan& p, cudaStream_t s);
cudaError_t launch_wide_chol_second(const Plan& p, double* R_out, int64_t ldr, cudaStream_t s);
cudaError_t launch_wide_jacobi(const Plan& p, const double* R, int64_t ldr, double* sigma, cudaStream_t s);
cudaError_t launch_svd_v(const Plan& p, const double* R, int64_t ldr, double* sigma, double* V, int64_t ldv,
                         cudaStream_t s);

}  // namespace figaro
