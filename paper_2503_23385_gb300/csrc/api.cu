// C ABI entry points (include/figaro.h): argument checks, workspace layout
// and the stream-ordered pipeline of one instance:
//   key grouping -> head/tail of A and B -> Gram pass 1 -> Cholesky 1 ->
//   Gram pass 2 -> Cholesky 2 and R = R2 R1 -> one-sided Jacobi.
#include <algorithm>
#include <array>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/figaro.h"
#include "common.cuh"
#include "internal.h"

namespace figaro {

int ht_chunk_rows(int n, int in_f64, int mixed);
void gram_geometry(int kout, int* kpad, int* ntiles, int* slices, int* tpt);

namespace {
std::atomic<int64_t> g_launches{0};
}  // namespace

void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {

struct Bump {
  char* base;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~static_cast<size_t>(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += sizeof(T) * (count > 0 ? count : 1);
    return p;
  }
};

int sm_count() {
  static std::mutex mu;
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  std::lock_guard<std::mutex> lock(mu);
  if (cache[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
    cache[dev] = v;
  }
  return cache[dev];
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

size_t plan_layout(Plan& p, const void* ws_base, int64_t m1, int n1, int64_t m2, int n2, int in_f64, int mixed,
                   int stage_a, int stage_b, int num_sms) {
  Bump b{static_cast<char*>(const_cast<void*>(ws_base))};
  p.n1 = n1;
  p.n2 = n2;
  p.n = n1 + n2;
  p.lut_size = (m1 > m2 ? m1 : m2) > 0 ? (m1 > m2 ? m1 : m2) : 1;
  p.mixed = mixed;
  p.num_sms = num_sms;
  const size_t ec = mixed ? 4 : 8;   // compute element
  const size_t ei = in_f64 ? 8 : 4;  // input element
  p.hdr = b.take<DevHeader>(1);
  int64_t ms[2] = {m1, m2};
  int ns[2] = {n1, n2};
  int stage[2] = {stage_a, stage_b};
  for (int t = 0; t < 2; ++t) {
    TableWork& T = p.t[t];
    const int64_t m = ms[t];
    const int n = ns[t];
    T.m = m;
    T.n = n;
    T.in_f64 = in_f64;
    if (stage[t]) {
      T.x = b.take<char>(static_cast<size_t>(m) * n * ei);
      T.key = b.take<int32_t>(static_cast<size_t>(m));
      T.ld = n;
    }
    T.tiles = static_cast<int>(ceil_div(m, kSortTile));
    for (int k = 0; k < 2; ++k) {
      T.kb[k] = b.take<uint32_t>(static_cast<size_t>(m));
      T.vb[k] = b.take<int32_t>(static_cast<size_t>(m));
    }
    T.hist = b.take<uint32_t>(static_cast<size_t>(kMaxPasses) * kRadixBins);
    T.sort_status = b.take<uint64_t>(static_cast<size_t>(group_status_words(T.tiles > 0 ? T.tiles : 1)));
    T.run_status = T.sort_status + static_cast<int64_t>(kMaxPasses) * (T.tiles > 0 ? T.tiles : 1) * kRadixBins;
    T.perm = b.take<int32_t>(static_cast<size_t>(m));
    T.sorted_key = b.take<int32_t>(static_cast<size_t>(m));
    T.seg = b.take<int32_t>(static_cast<size_t>(m));
    T.run_key = b.take<int32_t>(static_cast<size_t>(m));
    T.run_off = b.take<int32_t>(static_cast<size_t>(m) + 1);
    T.other = b.take<int32_t>(static_cast<size_t>(m));
    T.hdslot = b.take<int32_t>(static_cast<size_t>(m));
    T.run_info = b.take<int32_t>(static_cast<size_t>(m) * 4);
    T.lut = b.take<int32_t>(static_cast<size_t>(p.lut_size));
    T.tail = b.take<char>(static_cast<size_t>(m) * n * ec);
    T.chunk_rows = ht_chunk_rows(n, in_f64, mixed);
    T.chunks = static_cast<int>(ceil_div(m, T.chunk_rows));
    T.cbeg = b.take<int32_t>(static_cast<size_t>(T.chunks) + 1);
    T.cflag = b.take<uint32_t>(static_cast<size_t>(T.chunks));
    T.piece = b.take<double>(static_cast<size_t>(T.chunks) * n);
    T.carry = b.take<double>(static_cast<size_t>(T.chunks) * n);
  }
  const int n = p.n;
  p.head = b.take<char>(static_cast<size_t>(m1 > 0 ? m1 : 1) * n * ec);
  p.wide = n > kMaxWidth ? 1 : 0;
  // Gram partials, sized for the larger of the two passes
  for (int blk = 0; blk < 3; ++blk) {
    const int64_t rows = blk == 0 ? m1 : (blk == 1 ? m1 : m2);
    int64_t grid = ceil_div(rows, kGramTileRows);
    if (grid > 2 * num_sms) grid = 2 * num_sms;
    if (grid < 1) grid = 1;
    p.ggrid[blk] = static_cast<int>(grid);
    size_t most = 0;
    int kouts[2] = {blk == 0 ? n : (blk == 1 ? n1 : n2), blk == 2 ? n2 : n};
    for (int q = 0; q < 2; ++q) {
      size_t sz = static_cast<size_t>(grid) * kouts[q] * kouts[q];
      if (sz > most) most = sz;
    }
    // narrow mixed plans with n in (64, 128]: room for the tile Gram's
    // 128 x 128 partials of the head rows and of pass 2 on the A tails (one
    // per 1024 rows at most)
    if (blk <= 1 && !p.wide && mixed && n > 64 && n % 4 == 0) {
      const int64_t tiles = std::min<int64_t>(std::max<int64_t>(1, ceil_div(m1, 1024)), 2 * num_sms);
      most = std::max(most, static_cast<size_t>(tiles) * kWideTcTile * kWideTcTile);
    }
    p.gslices[blk] = 0;
    p.gcap[blk] = p.wide ? 1 : static_cast<int64_t>(most);
    p.gpart[blk] = b.take<double>(p.wide ? 1 : most);
  }
  if (p.wide) {
    const size_t qrows[3] = {static_cast<size_t>(m1), static_cast<size_t>(m1), static_cast<size_t>(m2)};
    const size_t qcols[3] = {static_cast<size_t>(n), static_cast<size_t>(n), static_cast<size_t>(n2)};
    for (int blk = 0; blk < 3; ++blk) p.wq[blk] = b.take<char>(qrows[blk] * qcols[blk] * ec);
    p.wpart = b.take<double>(static_cast<size_t>(wide_gram_part_doubles(m1, n1, m2, n2, num_sms, p.mixed)));
    if (p.mixed) {
      p.wt = b.take<float>(static_cast<size_t>(n) * n);
      p.wtlo = b.take<float>(static_cast<size_t>(n) * n);
    }
    const size_t nn = static_cast<size_t>(n) * n;
    p.Aw = b.take<char>(nn * ec);
    p.Tw = b.take<char>(nn * ec);
    p.Xw = b.take<double>(nn);
    p.yw = b.take<char>(static_cast<size_t>(n) * ec);
    p.d0w = b.take<char>(static_cast<size_t>(n) * ec);
  }
  // narrow mixed plans with n in (64, 128]: Q of the head rows and of the A
  // tails and W^T for the tensor-core formation and tile Gram of pass 2 (narrow_tc)
  if (!p.wide && mixed && n > 64 && n % 4 == 0) {
    p.wq[0] = b.take<char>(static_cast<size_t>(m1 > 0 ? m1 : 1) * n * 4);
    p.wq[1] = b.take<char>(static_cast<size_t>(m1 > 0 ? m1 : 1) * n * 4);
    p.wt = b.take<float>(static_cast<size_t>(n) * n);
    p.wtlo = b.take<float>(static_cast<size_t>(n) * n);
  }
  // the block Jacobi's columns (wide widths, and singular vectors at every width)
  p.Uw = b.take<char>(static_cast<size_t>(n + 32) * n * ec);
  p.Vw = b.take<char>(static_cast<size_t>(n + 32) * n * ec);
  p.sigw = b.take<double>(2 * static_cast<size_t>(n));  // Rayleigh quotients, column norms
  const size_t nn = static_cast<size_t>(n) * n;
  p.G1 = b.take<double>(nn);
  p.G2 = b.take<double>(nn);
  p.R1 = b.take<double>(nn);
  p.W = b.take<double>(nn);
  p.Wf = b.take<float>(nn);
  p.R = b.take<double>(nn);
  p.sigma = b.take<double>(static_cast<size_t>(n));
  p.active = b.take<int32_t>(static_cast<size_t>(n));
  return (b.off + 255) & ~static_cast<size_t>(255);
}

namespace {

// Library-owned side streams for staging host tables (created once per
// device; calls that stage at the same time share them, which orders their
// copies but never their results).
constexpr int kStageStreams = 4;
std::mutex g_stage_mu;
cudaStream_t g_stage_streams[64][kStageStreams] = {};

cudaError_t stage_streams(cudaStream_t (&out)[kStageStreams]) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_stage_mu);
  for (int i = 0; i < kStageStreams; ++i) {
    if (!g_stage_streams[dev][i]) {
      e = cudaStreamCreateWithFlags(&g_stage_streams[dev][i], cudaStreamNonBlocking);
      if (e != cudaSuccess) return e;
    }
    out[i] = g_stage_streams[dev][i];
  }
  return cudaSuccess;
}

struct Call {
  Plan p;
  cudaStream_t s = nullptr;
  cudaEvent_t ev[FIGARO_NUM_PHASE_EVENTS] = {};
  bool events = false;
  // host tables: the feature copies run on side streams while the call's
  // stream groups the keys; the call's stream waits for them (join_staging)
  // before the first step that reads features, table by table where the
  // head/tail step runs per table
  cudaEvent_t staged[kStageStreams] = {};
  int staged_table[kStageStreams] = {};
  int nstaged = 0;
  cudaError_t join_staging(int table = -1) {
    cudaError_t err = cudaSuccess;
    int kept = 0;
    for (int i = 0; i < nstaged; ++i) {
      if (table >= 0 && staged_table[i] != table) {
        staged[kept] = staged[i];
        staged_table[kept++] = staged_table[i];
        continue;
      }
      const cudaError_t e = cudaStreamWaitEvent(s, staged[i], 0);
      if (e != cudaSuccess && err == cudaSuccess) err = e;
      cudaEventDestroy(staged[i]);
    }
    nstaged = kept;
    return err;
  }
  bool staged_both() const {
    bool t0 = false, t1 = false;
    for (int i = 0; i < nstaged; ++i) (staged_table[i] ? t1 : t0) = true;
    return t0 && t1;
  }
  cudaError_t mark(int i) {
    if (!events) return cudaSuccess;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    // inside a stream capture the record must become an event node of the graph
    return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev[i], s, cudaEventRecordExternal)
                                               : cudaEventRecord(ev[i], s);
  }
};

figaro_status check_table(const figaro_table* T) {
  if (!T) return FIGARO_ERR_INVALID_ARG;
  if (T->m < 0 || T->m >= (int64_t{1} << 31)) return T->m < 0 ? FIGARO_ERR_INVALID_ARG : FIGARO_ERR_UNSUPPORTED;
  if (T->n < 1) return FIGARO_ERR_INVALID_ARG;
  if (T->ld < T->n) return FIGARO_ERR_INVALID_ARG;
  if (T->dtype != FIGARO_F32 && T->dtype != FIGARO_F64) return FIGARO_ERR_INVALID_ARG;
  if (T->memory != FIGARO_MEM_DEVICE && T->memory != FIGARO_MEM_HOST) return FIGARO_ERR_INVALID_ARG;
  if (T->m > 0 && (!T->x || !T->key)) return FIGARO_ERR_INVALID_ARG;
  return FIGARO_OK;
}

figaro_status check_pair(const figaro_table* A, const figaro_table* B, const figaro_options* o) {
  figaro_status st = check_table(A);
  if (st != FIGARO_OK) return st;
  st = check_table(B);
  if (st != FIGARO_OK) return st;
  if (A->dtype != B->dtype) return FIGARO_ERR_INVALID_ARG;
  if (o && o->path != FIGARO_PATH_FP64 && o->path != FIGARO_PATH_MIXED) return FIGARO_ERR_INVALID_ARG;
  if (o && (o->gram_engine < 0 || o->gram_engine > 2)) return FIGARO_ERR_INVALID_ARG;
  if (o && (o->max_jacobi_sweeps < 0 || o->spin_limit < 0 || !(o->rank_tol >= 0.0) || o->rank_tol >= 1.0))
    return FIGARO_ERR_INVALID_ARG;
  const int64_t n = static_cast<int64_t>(A->n) + B->n;
  if (n > kMaxWideWidth || (n > kMaxWidth && (A->n > kMaxTableWidth || B->n > kMaxTableWidth)))
    return FIGARO_ERR_UNSUPPORTED;
  return FIGARO_OK;
}

figaro_options resolve(const figaro_options* o) {
  figaro_options r;
  figaro_default_options(&r);
  if (o) r = *o;
  if (r.max_jacobi_sweeps == 0) r.max_jacobi_sweeps = 40;
  if (r.spin_limit == 0) r.spin_limit = 20000000;  // ~1-2 s of short naps
  return r;
}

// The device that owns the workspace becomes current for this thread.
figaro_status bind_device(const void* ws) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, ws) != cudaSuccess) {
    cudaGetLastError();
    return FIGARO_ERR_INVALID_ARG;
  }
  if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged) return FIGARO_ERR_INVALID_ARG;
  if (cudaSetDevice(attr.device) != cudaSuccess) return FIGARO_ERR_CUDA;
  return FIGARO_OK;
}

figaro_status prepare(Call& c, const figaro_table* A, const figaro_table* B, const figaro_options* opt, void* ws,
                      size_t ws_bytes, void* stream) {
  figaro_status st = check_pair(A, B, opt);
  if (st != FIGARO_OK) return st;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u)) return FIGARO_ERR_INVALID_ARG;
  st = bind_device(ws);
  if (st != FIGARO_OK) return st;
  figaro_options o = resolve(opt);
  const int in_f64 = A->dtype == FIGARO_F64;
  const int mixed = o.path == FIGARO_PATH_MIXED;
  const int sa = A->memory == FIGARO_MEM_HOST, sb = B->memory == FIGARO_MEM_HOST;
  size_t need = plan_layout(c.p, ws, A->m, A->n, B->m, B->n, in_f64, mixed, sa, sb, sm_count());
  if (ws_bytes < need) return FIGARO_ERR_WORKSPACE_TOO_SMALL;
  c.p.gram_engine = o.gram_engine;
  c.p.max_sweeps = o.max_jacobi_sweeps;
  c.p.spin_limit = o.spin_limit;
  c.p.rank_tol = o.rank_tol;
  c.p.withhold = (o.flags & FIGARO_FLAG_TEST_WITHHOLD) ? 1 : 0;
  c.p.report_rank = (o.flags & FIGARO_FLAG_ALLOW_RANK_DEFICIENT) ? 0 : c.p.n;
  c.p.shifted = (o.flags & FIGARO_FLAG_SHIFTED_CHOLQR3) ? 1 : 0;
  c.p.presorted = (o.flags & FIGARO_FLAG_PRESORTED) ? 1 : 0;
  c.p.sigma_dqds = (o.flags & FIGARO_FLAG_SIGMA_DQDS) ? 1 : 0;
  c.s = static_cast<cudaStream_t>(stream);
  if (o.phase_events) {
    c.events = true;
    for (int i = 0; i < FIGARO_NUM_PHASE_EVENTS; ++i) {
      c.ev[i] = static_cast<cudaEvent_t>(o.phase_events[i]);
      if (!c.ev[i]) return FIGARO_ERR_INVALID_ARG;
    }
  }
  const figaro_table* tabs[2] = {A, B};
  const size_t ei = in_f64 ? 8 : 4;
  bool staging = false;
  for (int t = 0; t < 2; ++t) {
    TableWork& T = c.p.t[t];
    const figaro_table* src = tabs[t];
    if (src->memory == FIGARO_MEM_HOST) {
      // the keys on the call's stream: key grouping needs nothing else
      if (src->m > 0) {
        if (cudaMemcpyAsync(const_cast<int32_t*>(T.key), src->key, sizeof(int32_t) * src->m, cudaMemcpyHostToDevice,
                            c.s) != cudaSuccess)
          return FIGARO_ERR_CUDA;
        staging = true;
      }
    } else {
      T.x = src->x;
      T.key = src->key;
      T.ld = src->ld;
    }
  }
  if (staging) {
    // the features in halves of each table on the side streams, after the
    // call's stream has reached this point (the staging area may still be
    // read by an earlier call on the same workspace)
    cudaStream_t ss[kStageStreams];
    cudaEvent_t fork = nullptr;
    if (stage_streams(ss) != cudaSuccess || cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(fork, c.s) != cudaSuccess)
      return FIGARO_ERR_CUDA;
    // (table B's copies start when table A's have landed: the link is shared,
    // so A arrives in half the time and its head/tail step overlaps B's copy)
    int part = 0;
    cudaError_t err = cudaSuccess;
    for (int t = 0; t < 2 && err == cudaSuccess; ++t) {
      const figaro_table* src = tabs[t];
      if (src->memory != FIGARO_MEM_HOST || src->m == 0) continue;
      TableWork& T = c.p.t[t];
      const int64_t half = (src->m + 1) / 2;
      const int earlier = c.nstaged;  // table A's copies, when t = 1
      for (int h = 0; h < 2 && err == cudaSuccess; ++h) {
        const int64_t r0 = h * half, r1 = h ? src->m : half;
        if (r1 <= r0) continue;
        cudaStream_t st = ss[part];
        cudaEvent_t done = nullptr;
        err = cudaStreamWaitEvent(st, fork, 0);
        for (int i = 0; i < earlier && err == cudaSuccess; ++i) err = cudaStreamWaitEvent(st, c.staged[i], 0);
        char* dst = static_cast<char*>(const_cast<void*>(T.x)) + static_cast<size_t>(r0) * src->n * ei;
        const char* from = static_cast<const char*>(src->x) + static_cast<size_t>(r0) * src->ld * ei;
        if (err == cudaSuccess && src->ld == src->n)  // dense rows: one contiguous copy
          err = cudaMemcpyAsync(dst, from, static_cast<size_t>(r1 - r0) * src->n * ei, cudaMemcpyHostToDevice, st);
        else if (err == cudaSuccess)
          err = cudaMemcpy2DAsync(dst, static_cast<size_t>(src->n) * ei, from, static_cast<size_t>(src->ld) * ei,
                                  static_cast<size_t>(src->n) * ei, static_cast<size_t>(r1 - r0), cudaMemcpyHostToDevice,
                                  st);
        if (err == cudaSuccess) err = cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
        if (err == cudaSuccess) err = cudaEventRecord(done, st);
        if (done) {
          c.staged_table[c.nstaged] = t;
          c.staged[c.nstaged++] = done;
        }
        ++part;
      }
    }
    cudaEventDestroy(fork);
    if (err != cudaSuccess) {
      c.join_staging();
      return FIGARO_ERR_CUDA;
    }
  }
  return FIGARO_OK;
}

// Joins a call's staging copies into its stream when the entry point returns
// (also on an early error return, so no copy is left unordered).
struct StageJoin {
  Call& c;
  ~StageJoin() { c.join_staging(); }
};

#define FIGARO_TRY(expr)                                   \
  do {                                                     \
    cudaError_t e_ = (expr);                               \
    if (e_ != cudaSuccess) return FIGARO_ERR_CUDA;         \
  } while (0)

figaro_status run_grouping(Call& c) {
  FIGARO_TRY(c.mark(0));
  FIGARO_TRY(launch_reset(c.p, c.s));
  FIGARO_TRY(launch_grouping(c.p, c.s));
  FIGARO_TRY(c.mark(1));
  return FIGARO_OK;
}

figaro_status run_factor(Call& c, double* R_dev, int64_t ldr) {
  // both tables staged from host memory: the head/tail step runs per table,
  // each as its features land
  c.p.ht_split = c.staged_both() ? 1 : 0;
  ht_plan_gram1(c.p);  // pass 1 of the tail blocks inside the head/tail stream, where it applies
  if (c.p.ht_split) {
    for (int t = 0; t < 2; ++t) {
      FIGARO_TRY(c.join_staging(t));
      FIGARO_TRY(launch_ht_carry(c.p, c.s, t));
      if (t == 0) FIGARO_TRY(c.mark(2));
      FIGARO_TRY(launch_ht_main(c.p, c.s, t));
    }
  } else {
    FIGARO_TRY(c.join_staging());  // the features are read from here on
    FIGARO_TRY(launch_ht_carry(c.p, c.s));
    FIGARO_TRY(c.mark(2));
    FIGARO_TRY(launch_ht_main(c.p, c.s));
  }
  FIGARO_TRY(c.mark(3));
  FIGARO_TRY(launch_gram_pass(c.p, 1, c.s));
  FIGARO_TRY(c.mark(4));
  FIGARO_TRY(launch_chol_first(c.p, c.s));
  FIGARO_TRY(c.mark(5));
  FIGARO_TRY(launch_gram_pass(c.p, 2, c.s));
  FIGARO_TRY(c.mark(6));
  if (c.p.shifted) {
    // shifted CholeskyQR3: the shifted first pass leaves Q = M R1^{-1} with a
    // moderate condition number; the factor R' = R2 R1 of the second pass
    // preconditions a third pass (W = R'^{-1}, Gram of M W, R = R3 R')
    FIGARO_TRY(launch_chol_second(c.p, nullptr, ldr, c.s));
    FIGARO_TRY(launch_refactor(c.p, c.s));
    FIGARO_TRY(launch_gram_pass(c.p, 2, c.s));
  }
  FIGARO_TRY(launch_chol_second(c.p, R_dev, ldr, c.s));
  FIGARO_TRY(c.mark(7));
  return FIGARO_OK;
}

figaro_status run_qr_svd(Call& c, double* R_out, int64_t ldr, double* sigma, int host_out) {
  figaro_status st = run_grouping(c);
  if (st != FIGARO_OK) return st;
  const int n = c.p.n;
  st = run_factor(c, host_out ? nullptr : R_out, ldr);
  if (st != FIGARO_OK) return st;
  if (sigma) {
    double* sg = host_out ? c.p.sigma : sigma;
    FIGARO_TRY(c.p.sigma_dqds ? launch_sigma_dqds(c.p, c.p.R, n, sg, c.s) : launch_jacobi(c.p, c.p.R, n, sg, c.s));
  }
  FIGARO_TRY(c.mark(8));
  if (host_out) {
    if (R_out)
      FIGARO_TRY(cudaMemcpy2DAsync(R_out, sizeof(double) * ldr, c.p.R, sizeof(double) * n, sizeof(double) * n, n,
                                   cudaMemcpyDeviceToHost, c.s));
    if (sigma) FIGARO_TRY(cudaMemcpyAsync(sigma, c.p.sigma, sizeof(double) * n, cudaMemcpyDeviceToHost, c.s));
  }
  return FIGARO_OK;
}

// Library-owned scratch of figaro_join_singular_values_fixed (a fixed-size
// device array, so the call needs no allocation).  In host code the array's
// name is not a device address: every call asks the runtime for the address
// of the current device's copy (a host-side query that allocates nothing).
// The address is not cached, because it belongs to the context the
// library's device code was loaded into: after a cudaDeviceReset, or in
// another context, the module is loaded again and the array can move.
__device__ __align__(256) unsigned char g_fixed_scratch[FIGARO_FIXED_SCRATCH_BYTES];

figaro_status fixed_scratch(void** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_fixed_scratch) != cudaSuccess || !p) {
    cudaGetLastError();
    return FIGARO_ERR_CUDA;
  }
  *out = p;
  return FIGARO_OK;
}

// The device of the first non-empty device-resident table becomes current.
figaro_status bind_input_device(const figaro_table* A, const figaro_table* B) {
  const figaro_table* tabs[2] = {A, B};
  for (const figaro_table* T : tabs)
    if (T->memory == FIGARO_MEM_DEVICE && T->m > 0) return bind_device(T->x);
  return FIGARO_OK;
}


// ------------------------------------------------------------- batching ----
//
// figaro_batch_join runs every narrow, device-resident instance of a batch
// with one launch per phase: the per-instance plans and, per launch, a job
// list (job -> instance, CTAs) are built on the host, written into the front
// of the workspace by copy kernels whose arguments carry the bytes (so the
// whole call can be captured in a CUDA graph), and each batched kernel maps
// its CTA to (instance, CTA within the job).

constexpr int kUploadBytes = 30 * 1024;  // kernel arguments of up to 32,764 bytes

struct UploadChunk {
  unsigned char* dst;
  int bytes;
  int pad[1];
  alignas(16) unsigned char data[kUploadBytes];
};

__global__ void upload_kernel(const __grid_constant__ UploadChunk c) {
  pdl_enter();
  // 16-byte words where the destination allows, then the bytes of the tail
  const int nv = (reinterpret_cast<uintptr_t>(c.dst) & 15) == 0 ? c.bytes / 16 : 0;
  const uint4* src = reinterpret_cast<const uint4*>(c.data);
  uint4* dst = reinterpret_cast<uint4*>(c.dst);
  for (int i = threadIdx.x; i < nv; i += blockDim.x) dst[i] = src[i];
  for (int i = 16 * nv + static_cast<int>(threadIdx.x); i < c.bytes; i += blockDim.x) c.dst[i] = c.data[i];
}

// Bytes of the batch area (plans, outputs, job lists) for `count` instances.
size_t batch_area_bytes(int count) {
  const size_t lists = 24, per_list = (3 * static_cast<size_t>(count) + 1) * 3 * sizeof(int32_t) + 256;
  // the table launches of the wide tensor-core kernels: per instance at most
  // three tile-Gram entries, two formation entries, one W^T entry and their
  // CTA offsets
  const size_t tables = (3 * sizeof(WideTcEntry) + 2 * sizeof(WideFormEntry) + sizeof(WidePrepEntry) +
                         6 * sizeof(int32_t)) * static_cast<size_t>(count) + 12 * 128;
  // per pass the jobs' Gram arguments (three blocks) and reduce arguments of every instance
  const size_t args = 2 * (3 * batch_gram_args_bytes() + batch_reduce_args_bytes()) * static_cast<size_t>(count) + 512;
  return ((sizeof(Plan) + sizeof(BatchOut)) * static_cast<size_t>(count) + lists * per_list + tables + args + 4096 +
          255) & ~static_cast<size_t>(255);
}

struct JobList {
  std::vector<int32_t> first{0}, inst, aux;
  void add(int i, int a, int ctas) {
    if (ctas <= 0) return;
    inst.push_back(i);
    aux.push_back(a);
    first.push_back(first.back() + ctas);
  }
  int njobs() const { return static_cast<int>(inst.size()); }
};

struct Blob {
  std::vector<unsigned char> bytes;
  size_t put(const void* src, size_t n, size_t align = 16) {
    size_t off = (bytes.size() + align - 1) & ~(align - 1);
    bytes.resize(off + n);
    if (n) std::memcpy(bytes.data() + off, src, n);
    return off;
  }
};

BatchJobs stage_jobs(Blob& blob, const JobList& L, std::vector<std::pair<BatchJobs*, size_t[3]>>& fix, BatchJobs* dst) {
  BatchJobs J{};
  J.njobs = L.njobs();
  J.ctas = L.first.back();
  fix.emplace_back();
  fix.back().first = dst;
  fix.back().second[0] = blob.put(L.first.data(), L.first.size() * sizeof(int32_t));
  fix.back().second[1] = blob.put(L.inst.data(), L.inst.size() * sizeof(int32_t));
  fix.back().second[2] = blob.put(L.aux.data(), L.aux.size() * sizeof(int32_t));
  return J;
}

// The schedule of a batched call: rows of a Gram block per CTA, and the
// head/tail CTA budget in multiples of the SM count.
struct BatchSchedule {
  int64_t gram_rows_per_cta = 4096;
  int ht_ctas_per_sm = 2;
};

figaro_status run_batched(std::vector<Call>& calls, const std::vector<BatchOut>& outs, char* area, size_t area_bytes,
                          cudaStream_t s, void* const* phase_events, const BatchSchedule& sched) {
  const int count = static_cast<int>(calls.size());
  if (count == 0) return FIGARO_OK;
  // Gram grids from the schedule (never above the partial buffers the plans reserved)
  std::vector<std::array<int, 3>> grid0(calls.size());
  for (size_t i = 0; i < calls.size(); ++i)
    for (int b = 0; b < 3; ++b) grid0[i][b] = calls[i].p.ggrid[b];
  for (Call& c : calls) {
    const int64_t rows[3] = {c.p.t[0].m, c.p.t[0].m, c.p.t[1].m};
    for (int b = 0; b < 3; ++b) {
      const int64_t g = (rows[b] + sched.gram_rows_per_cta - 1) / sched.gram_rows_per_cta;
      c.p.ggrid[b] = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(g, c.p.ggrid[b])));
    }
  }
  const Plan& p0 = calls[0].p;
  const int mixed = p0.mixed, in_f64 = p0.t[0].in_f64;
  // ---- job lists
  JobList tiles, match, htplan, htscan, htstream[2], gram[2][4], reduce, dense1[3], dense2[3], dense3[3];
  std::vector<TcJob> tc[2][2][4];  // [pass][engine - 1][variant]
  size_t tc_smem[2][2][4] = {};
  int ht_smem[2] = {0, 0};
  size_t gram_smem[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
  size_t dsm[3][3] = {};
  int dthr[3][3] = {};
  // blocks with n in (64, 128] output columns on the mixed path (the head
  // rows in both passes, the A tails in pass 2): per pass, table launches of
  // the W^T preparation, the tensor-core formation and the tile Gram
  // (entries 128-byte aligned in the batch area)
  struct QTables {
    std::vector<WideTcEntry> t;
    std::vector<WideFormEntry> f;
    std::vector<WidePrepEntry> w;
    std::vector<int32_t> t0{0}, f0{0}, w0{0};
    size_t off_t = 0, off_f = 0, off_w = 0, off_t0 = 0, off_f0 = 0, off_w0 = 0;
  } qtab[2];
  const bool q_tables = (reinterpret_cast<uintptr_t>(area) & 127) == 0;
  int64_t total_chunks = 0;
  for (int i = 0; i < count; ++i)
    for (int t = 0; t < 2; ++t) total_chunks += calls[i].p.t[t].m > 0 ? calls[i].p.t[t].chunks : 0;
  const int64_t gtot = static_cast<int64_t>(sched.ht_ctas_per_sm) * p0.num_sms;
  for (int i = 0; i < count; ++i) {
    const Plan& p = calls[i].p;
    for (int t = 0; t < 2; ++t) {
      tiles.add(i, t, p.t[t].tiles);
      int v = 0, sm = 0, chunks = 0;
      ht_batch_table(p, t, &v, &sm, &chunks);
      if (chunks == 0) continue;
      htplan.add(i, t, chunks);
      htscan.add(i, t, p.t[t].n);
      int64_t g = (static_cast<int64_t>(chunks) * gtot + total_chunks - 1) / total_chunks;
      g = std::max<int64_t>(1, std::min<int64_t>(g, chunks));
      htstream[v].add(i, t, static_cast<int>(g));
      ht_smem[v] = std::max(ht_smem[v], sm);
    }
    const int64_t mm = std::max(p.t[0].m, p.t[1].m);
    match.add(i, 0, static_cast<int>((mm + 255) / 256));
    bool prep_added = false;
    for (int pass = 1; pass <= 2; ++pass)
      for (int b = 0; b < 3; ++b) {
        if (q_tables && narrow_tc(p, pass, b)) {
          WideFormBlock fb;
          WideTcBlock tb;
          narrow_tc_blocks(p, pass, b, sched.gram_rows_per_cta, &fb, &tb);
          WideFormEntry fe;
          WideTcEntry te;
          if ((pass == 1 || wide_form_encode(fb, &fe)) && wide_tc_encode(tb, &te)) {
            QTables& Q = qtab[pass - 1];
            if (pass == 2) {
              Q.f.push_back(fe);
              Q.f0.push_back(Q.f0.back() + fb.njobs);
              if (!prep_added) {
                Q.w.push_back(WidePrepEntry{p.Wf, p.wt, p.wtlo, p.n});
                Q.w0.push_back(Q.w0.back() + (p.n * p.n + 255) / 256);
                prep_added = true;
              }
            }
            Q.t.push_back(te);
            Q.t0.push_back(Q.t0.back() + tb.njobs);
            calls[i].p.gcount[pass - 1][b] = tb.njobs;
            calls[i].p.gsym[pass - 1][b] = 3;
            continue;
          }
        }
        int tv = 0;
        int64_t tile_rows = 0;
        size_t tsm = 0;
        const int eng = gram_tc_batch_engine(p, pass, b, &tv, &tile_rows, &tsm);
        if (eng > 0) {  // tensor cores: CTAs by the schedule's rows per CTA
          const int64_t rows = b == 2 ? p.t[1].m : p.t[0].m;
          const int64_t per = std::max<int64_t>(sched.gram_rows_per_cta, tile_rows);
          const int ctas = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((rows + per - 1) / per, grid0[i][b])));
          tc[pass - 1][eng - 1][tv].push_back(TcJob{i, b, ctas});
          tc_smem[pass - 1][eng - 1][tv] = std::max(tc_smem[pass - 1][eng - 1][tv], tsm);
          calls[i].p.gcount[pass - 1][b] = ctas;
          calls[i].p.gsym[pass - 1][b] = eng == 2 ? 1 : 2;  // general engine: P pairs; packed: float-float
          continue;
        }
        int v = 0, ctas = 0;
        size_t sm = 0;
        gram_batch_block(p, pass, b, &v, &ctas, &sm);
        if (ctas == 0) continue;
        gram[pass - 1][v].add(i, b, ctas);
        gram_smem[pass - 1][v] = std::max(gram_smem[pass - 1][v], sm);
        calls[i].p.gcount[pass - 1][b] = ctas;
        calls[i].p.gsym[pass - 1][b] = 0;
      }
    // the reduce: a warp per 32 outputs when every block has few partials
    int most = 0;
    for (int q = 0; q < 2; ++q)
      for (int b = 0; b < 3; ++b) most = std::max(most, p.gcount[q][b] > 0 ? p.gcount[q][b] : p.ggrid[b]);
    if (most <= 64) reduce.add(i, 1, (p.n * p.n + 32 * kReduceWarps - 1) / (32 * kReduceWarps));
    else reduce.add(i, 0, (p.n * p.n + 31) / 32);
  }
  // the n x n steps: one CTA per instance, the widest instances first (their
  // CTAs take longest, so the others fill in around them)
  std::vector<int> by_width(count);
  for (int i = 0; i < count; ++i) by_width[i] = i;
  std::stable_sort(by_width.begin(), by_width.end(), [&](int a, int b) { return calls[a].p.n > calls[b].p.n; });
  for (int i : by_width) {
    const Plan& p = calls[i].p;
    JobList* dl[3] = {dense1, dense2, dense3};
    for (int step = 1; step <= 3; ++step) {
      if (step == 3 && !outs[i].sigma) continue;
      int v = 0, thr = 0;
      size_t sm = 0;
      if (step == 3 && p.sigma_dqds) {
        sm = sigma_dqds_smem(p.n, p.mixed);
        thr = sigma_dqds_threads();
      } else {
        dense_batch_info(p, step, &v, &sm, &thr);
      }
      dl[step - 1][v].add(i, 0, 1);
      dsm[step - 1][v] = std::max(dsm[step - 1][v], sm);
      dthr[step - 1][v] = std::max(dthr[step - 1][v], thr);
    }
  }
  // ---- the batch area: plans, outputs, job lists
  Blob blob;
  std::vector<Plan> plans(count);
  for (int i = 0; i < count; ++i) plans[i] = calls[i].p;
  const size_t off_plans = blob.put(plans.data(), sizeof(Plan) * count);
  const size_t off_outs = blob.put(outs.data(), sizeof(BatchOut) * count);
  std::vector<std::pair<BatchJobs*, size_t[3]>> fix;
  BatchJobs Jtiles, Jmatch, Jplan, Jscan, Jstream[2], Jgram[2][4], Jreduce, Jd[3][3];
  Jtiles = stage_jobs(blob, tiles, fix, &Jtiles);
  Jmatch = stage_jobs(blob, match, fix, &Jmatch);
  Jplan = stage_jobs(blob, htplan, fix, &Jplan);
  Jscan = stage_jobs(blob, htscan, fix, &Jscan);
  for (int v = 0; v < 2; ++v) Jstream[v] = stage_jobs(blob, htstream[v], fix, &Jstream[v]);
  for (int q = 0; q < 2; ++q)
    for (int v = 0; v < 4; ++v) Jgram[q][v] = stage_jobs(blob, gram[q][v], fix, &Jgram[q][v]);
  Jreduce = stage_jobs(blob, reduce, fix, &Jreduce);
  for (QTables& Q : qtab) {
    if (!Q.t.empty()) {
      Q.off_t = blob.put(Q.t.data(), sizeof(WideTcEntry) * Q.t.size(), 128);
      Q.off_t0 = blob.put(Q.t0.data(), sizeof(int32_t) * Q.t0.size());
    }
    if (!Q.f.empty()) {
      Q.off_f = blob.put(Q.f.data(), sizeof(WideFormEntry) * Q.f.size(), 128);
      Q.off_f0 = blob.put(Q.f0.data(), sizeof(int32_t) * Q.f0.size());
    }
    if (!Q.w.empty()) {
      Q.off_w = blob.put(Q.w.data(), sizeof(WidePrepEntry) * Q.w.size());
      Q.off_w0 = blob.put(Q.w0.data(), sizeof(int32_t) * Q.w0.size());
    }
  }
  JobList* dl[3] = {dense1, dense2, dense3};
  for (int st = 0; st < 3; ++st)
    for (int v = 0; v < 3; ++v) Jd[st][v] = stage_jobs(blob, dl[st][v], fix, &Jd[st][v]);
  // after the uploaded part: per pass the jobs' Gram and reduce arguments,
  // written on the device at the start of each Gram pass
  const size_t gab = batch_gram_args_bytes() * 3 * count, rab = batch_reduce_args_bytes() * count;
  const size_t off_args = (blob.bytes.size() + 255) & ~static_cast<size_t>(255);
  size_t off_gargs[2], off_rargs[2];
  for (int q = 0; q < 2; ++q) {
    off_gargs[q] = off_args + q * (gab + rab + 16);
    off_rargs[q] = (off_gargs[q] + gab + 15) & ~static_cast<size_t>(15);
  }
  if (blob.bytes.size() > area_bytes || off_rargs[1] + rab > area_bytes) return FIGARO_ERR_WORKSPACE_TOO_SMALL;
  for (auto& f : fix) {
    f.first->first = reinterpret_cast<const int32_t*>(area + f.second[0]);
    f.first->inst = reinterpret_cast<const int32_t*>(area + f.second[1]);
    f.first->aux = reinterpret_cast<const int32_t*>(area + f.second[2]);
  }
  for (size_t o = 0; o < blob.bytes.size(); o += kUploadBytes) {
    UploadChunk c;
    c.dst = reinterpret_cast<unsigned char*>(area) + o;
    c.bytes = static_cast<int>(std::min<size_t>(kUploadBytes, blob.bytes.size() - o));
    std::memcpy(c.data, blob.bytes.data() + o, c.bytes);
    pdl_launch(upload_kernel, 1, 512, 0, s, c);
    count_launches(1);
  }
  FIGARO_TRY(cudaGetLastError());
  BatchDev b;
  b.plans = reinterpret_cast<const Plan*>(area + off_plans);
  b.out = reinterpret_cast<const BatchOut*>(area + off_outs);
  b.count = count;
  // ---- the phases (with the phase events of single calls; the head/tail
  // carry and streaming launches share one interval)
  Call ev;
  ev.s = s;
  if (phase_events) {
    ev.events = true;
    for (int i = 0; i < FIGARO_NUM_PHASE_EVENTS; ++i) ev.ev[i] = static_cast<cudaEvent_t>(phase_events[i]);
  }
  FIGARO_TRY(ev.mark(0));
  FIGARO_TRY(launch_batch_grouping(b, Jtiles, Jmatch, s));
  FIGARO_TRY(ev.mark(1));
  FIGARO_TRY(ev.mark(2));
  FIGARO_TRY(launch_batch_ht(b, Jplan, Jplan.ctas, Jscan, Jstream, ht_smem, in_f64, mixed, s));
  FIGARO_TRY(ev.mark(3));
  const BatchJobs none[4] = {};
  const size_t none_smem[4] = {0, 0, 0, 0};
  auto gram_pass = [&](int pass) -> figaro_status {
    const BatchJobs empty{};
    void* gargs = area + off_gargs[pass - 1];
    void* rargs = area + off_rargs[pass - 1];
    FIGARO_TRY(launch_batch_args(b, pass, gargs, rargs, s));
    FIGARO_TRY(launch_batch_gram(b, pass, Jgram[pass - 1], gram_smem[pass - 1], empty, mixed, gargs, rargs, s));
    for (int e = 0; e < 2; ++e)
      for (int v = 0; v < 4; ++v) {
        const auto& jobs = tc[pass - 1][e][v];
        FIGARO_TRY(launch_gram_tc_batch(b.plans, plans.data(), pass, e + 1, v, jobs.data(), static_cast<int>(jobs.size()),
                                        tc_smem[pass - 1][e][v], s));
      }
    const QTables& Q = qtab[pass - 1];
    if (!Q.t.empty()) {  // (pass 2: W^T of each instance and Q = X W first) the tile Gram
      auto at = [&](size_t off) { return area + off; };
      if (!Q.w.empty())
        FIGARO_TRY(launch_wide_prep_table(reinterpret_cast<const WidePrepEntry*>(at(Q.off_w)),
                                          reinterpret_cast<const int32_t*>(at(Q.off_w0)),
                                          static_cast<int>(Q.w.size()), Q.w0.back(), s));
      if (!Q.f.empty())
        FIGARO_TRY(launch_wide_form_tc_table(reinterpret_cast<const WideFormEntry*>(at(Q.off_f)),
                                             reinterpret_cast<const int32_t*>(at(Q.off_f0)),
                                             static_cast<int>(Q.f.size()), Q.f0.back(), p0.spin_limit, s));
      FIGARO_TRY(launch_wide_gram_tc_table(reinterpret_cast<const WideTcEntry*>(at(Q.off_t)),
                                           reinterpret_cast<const int32_t*>(at(Q.off_t0)),
                                           static_cast<int>(Q.t.size()), Q.t0.back(), p0.spin_limit, s));
    }
    FIGARO_TRY(launch_batch_gram(b, pass, none, none_smem, Jreduce, mixed, gargs, rargs, s));
    return FIGARO_OK;
  };
  figaro_status gs = gram_pass(1);
  if (gs != FIGARO_OK) return gs;
  FIGARO_TRY(ev.mark(4));
  FIGARO_TRY(launch_batch_dense(b, 1, Jd[0], dsm[0], dthr[0], mixed, s));
  FIGARO_TRY(ev.mark(5));
  gs = gram_pass(2);
  if (gs != FIGARO_OK) return gs;
  FIGARO_TRY(ev.mark(6));
  FIGARO_TRY(launch_batch_dense(b, 2, Jd[1], dsm[1], dthr[1], mixed, s));
  FIGARO_TRY(ev.mark(7));
  if (calls[0].p.sigma_dqds)
    FIGARO_TRY(launch_batch_sigma_dqds(b, Jd[2][0], dsm[2][0], mixed, s));
  else
    FIGARO_TRY(launch_batch_dense(b, 3, Jd[2], dsm[2], dthr[2], mixed, s));
  FIGARO_TRY(ev.mark(8));
  return FIGARO_OK;
}


// ------------------------------------------------------------ autotuner ----
//
// A batch's schedule is chosen by timing candidates on the batch itself
// (FIGARO_FLAG_AUTOTUNE, outside stream capture): rows per Gram CTA from
// {1024, ..., 32768} with the Gram passes timed, then head/tail CTA budgets
// of {1, 2, 4, 8} x the SM count with the head/tail phase timed.  The
// fastest values are kept in a process-wide cache keyed by the batch's
// shape class (instances, path, input rows and summed widths, each rounded
// to a power of two) and used by every later call of that class.

struct TuneKey {
  int count, path, in_f64;
  int rows_log2, width_log2;
  bool operator<(const TuneKey& o) const {
    return std::tie(count, path, in_f64, rows_log2, width_log2) <
           std::tie(o.count, o.path, o.in_f64, o.rows_log2, o.width_log2);
  }
};

std::mutex g_tune_mu;
std::map<TuneKey, BatchSchedule> g_tuned;

int ilog2(int64_t v) {
  int r = 0;
  while (v > 1) {
    v >>= 1;
    ++r;
  }
  return r;
}

TuneKey tune_key(const std::vector<Call>& calls) {
  int64_t rows = 0, widths = 0;
  for (const Call& c : calls) {
    rows += c.p.t[0].m + c.p.t[1].m;
    widths += c.p.n;
  }
  TuneKey k{};
  k.count = static_cast<int>(calls.size());
  k.path = calls.empty() ? 0 : calls[0].p.mixed;
  k.in_f64 = calls.empty() ? 0 : calls[0].p.t[0].in_f64;
  k.rows_log2 = ilog2(rows + 1);
  k.width_log2 = ilog2(widths + 1);
  return k;
}

// Milliseconds between phase events a and b of one batched run.
figaro_status time_batched(std::vector<Call> calls, const std::vector<BatchOut>& outs, char* area, size_t area_bytes,
                           cudaStream_t s, const BatchSchedule& sched, int a, int b, float* ms) {
  cudaEvent_t ev[FIGARO_NUM_PHASE_EVENTS];
  for (int i = 0; i < FIGARO_NUM_PHASE_EVENTS; ++i)
    if (cudaEventCreate(&ev[i]) != cudaSuccess) return FIGARO_ERR_CUDA;
  void* evp[FIGARO_NUM_PHASE_EVENTS];
  for (int i = 0; i < FIGARO_NUM_PHASE_EVENTS; ++i) evp[i] = ev[i];
  figaro_status st = run_batched(calls, outs, area, area_bytes, s, evp, sched);
  if (st == FIGARO_OK && cudaStreamSynchronize(s) != cudaSuccess) st = FIGARO_ERR_CUDA;
  if (st == FIGARO_OK && cudaEventElapsedTime(ms, ev[a], ev[b]) != cudaSuccess) st = FIGARO_ERR_CUDA;
  for (int i = 0; i < FIGARO_NUM_PHASE_EVENTS; ++i) cudaEventDestroy(ev[i]);
  return st;
}

figaro_status tune_batch(const std::vector<Call>& calls, const std::vector<BatchOut>& outs, char* area,
                         size_t area_bytes, cudaStream_t s, BatchSchedule* best) {
  BatchSchedule cur;
  // warm the kernels once so that no candidate pays first-launch costs
  float ms = 0.f;
  figaro_status st = time_batched(calls, outs, area, area_bytes, s, cur, 0, 8, &ms);
  if (st != FIGARO_OK) return st;
  float best_ms = 1e30f;
  for (int64_t rpc = 1024; rpc <= 32768; rpc *= 2) {
    BatchSchedule c = cur;
    c.gram_rows_per_cta = rpc;
    float g1 = 0.f, g2 = 0.f;
    st = time_batched(calls, outs, area, area_bytes, s, c, 3, 4, &g1);
    if (st == FIGARO_OK) st = time_batched(calls, outs, area, area_bytes, s, c, 5, 6, &g2);
    if (st != FIGARO_OK) return st;
    if (g1 + g2 < best_ms) {
      best_ms = g1 + g2;
      cur.gram_rows_per_cta = rpc;
    }
  }
  best_ms = 1e30f;
  const int ht_candidates[4] = {1, 2, 4, 8};
  for (int h : ht_candidates) {
    BatchSchedule c = cur;
    c.ht_ctas_per_sm = h;
    float t = 0.f;
    st = time_batched(calls, outs, area, area_bytes, s, c, 2, 3, &t);
    if (st != FIGARO_OK) return st;
    if (t < best_ms) {
      best_ms = t;
      cur.ht_ctas_per_sm = h;
    }
  }
  *best = cur;
  return FIGARO_OK;
}

BatchSchedule schedule_for(const std::vector<Call>& calls) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tuned.find(tune_key(calls));
  return it == g_tuned.end() ? BatchSchedule{} : it->second;
}
}  // namespace
}  // namespace figaro

using namespace figaro;

extern "C" {

figaro_status figaro_default_options(figaro_options* opt) {
  if (!opt) return FIGARO_ERR_INVALID_ARG;
  std::memset(opt, 0, sizeof(*opt));
  opt->path = FIGARO_PATH_MIXED;
  opt->gram_engine = FIGARO_GRAM_AUTO;
  return FIGARO_OK;
}

figaro_status figaro_workspace_size(const figaro_table* A, const figaro_table* B, const figaro_options* opt,
                                    size_t* bytes) {
  if (!bytes) return FIGARO_ERR_INVALID_ARG;
  figaro_status st = check_pair(A, B, opt);
  if (st != FIGARO_OK) return st;
  figaro_options o = resolve(opt);
  Plan p;
  *bytes = plan_layout(p, nullptr, A->m, A->n, B->m, B->n, A->dtype == FIGARO_F64, o.path == FIGARO_PATH_MIXED,
                       A->memory == FIGARO_MEM_HOST, B->memory == FIGARO_MEM_HOST, sm_count());
  return FIGARO_OK;
}

figaro_status figaro_join_group(const figaro_table* A, const figaro_table* B, const figaro_options* opt,
                                const figaro_grouping* outA, const figaro_grouping* outB, int64_t* num_groups,
                                void* ws, size_t ws_bytes, void* stream) {
  if (!outA || !outB) return FIGARO_ERR_INVALID_ARG;
  const figaro_grouping* outs[2] = {outA, outB};
  const int64_t ms[2] = {A ? A->m : 0, B ? B->m : 0};
  for (int t = 0; t < 2; ++t) {
    const figaro_grouping* g = outs[t];
    if (!g->num_runs) return FIGARO_ERR_INVALID_ARG;
    if (ms[t] > 0 && (!g->perm || !g->sorted_key || !g->run_key || !g->run_offset || !g->other_count))
      return FIGARO_ERR_INVALID_ARG;
    if (!g->run_offset) return FIGARO_ERR_INVALID_ARG;
  }
  Call c;
  StageJoin join_at_exit{c};
  figaro_status st = prepare(c, A, B, opt, ws, ws_bytes, stream);
  if (st != FIGARO_OK) return st;
  for (int t = 0; t < 2; ++t) {
    TableWork& T = c.p.t[t];
    const figaro_grouping* g = outs[t];
    if (T.m > 0) {
      T.perm = g->perm;
      T.sorted_key = g->sorted_key;
      T.run_key = g->run_key;
      T.run_off = g->run_offset;
      T.other = g->other_count;
    }
  }
  st = run_grouping(c);
  if (st != FIGARO_OK) return st;
  for (int t = 0; t < 2; ++t) {
    FIGARO_TRY(cudaMemcpyAsync(outs[t]->num_runs, &c.p.hdr->num_runs[t], sizeof(int64_t), cudaMemcpyDeviceToDevice,
                               c.s));
    if (c.p.t[t].m == 0) FIGARO_TRY(cudaMemsetAsync(outs[t]->run_offset, 0, sizeof(int32_t), c.s));
  }
  if (num_groups)
    FIGARO_TRY(cudaMemcpyAsync(num_groups, &c.p.hdr->num_groups, sizeof(int64_t), cudaMemcpyDeviceToDevice, c.s));
  return FIGARO_OK;
}

figaro_status figaro_join_head_tail(const figaro_table* A, const figaro_table* B, const figaro_options* opt,
                                    void* head, void* tail_a, void* tail_b, void* ws, size_t ws_bytes,
                                    void* stream) {
  Call c;
  StageJoin join_at_exit{c};
  figaro_status st = prepare(c, A, B, opt, ws, ws_bytes, stream);
  if (st != FIGARO_OK) return st;
  if ((A->m > 0 && (!head || !tail_a)) || (B->m > 0 && !tail_b)) return FIGARO_ERR_INVALID_ARG;
  if (A->m > 0) {
    c.p.head = head;
    c.p.t[0].tail = tail_a;
  }
  if (B->m > 0) c.p.t[1].tail = tail_b;
  st = run_grouping(c);
  if (st != FIGARO_OK) return st;
  FIGARO_TRY(c.join_staging());
  FIGARO_TRY(launch_ht_carry(c.p, c.s));
  FIGARO_TRY(launch_ht_main(c.p, c.s));
  return FIGARO_OK;
}

figaro_status figaro_join_qr_r(const figaro_table* A, const figaro_table* B, const figaro_options* opt, double* R,
                               int64_t ldr, void* ws, size_t ws_bytes, void* stream) {
  if (!R) return FIGARO_ERR_INVALID_ARG;
  Call c;
  StageJoin join_at_exit{c};
  figaro_status st = prepare(c, A, B, opt, ws, ws_bytes, stream);
  if (st != FIGARO_OK) return st;
  if (ldr < c.p.n) return FIGARO_ERR_INVALID_ARG;
  const int host_out = opt && (opt->flags & FIGARO_FLAG_HOST_OUTPUT);
  return run_qr_svd(c, R, ldr, nullptr, host_out);
}

figaro_status figaro_join_singular_values(const figaro_table* A, const figaro_table* B, const figaro_options* opt,
                                          double* sigma, double* R_out, int64_t ldr, void* ws, size_t ws_bytes,
                                          void* stream) {
  if (!sigma) return FIGARO_ERR_INVALID_ARG;
  Call c;
  StageJoin join_at_exit{c};
  figaro_status st = prepare(c, A, B, opt, ws, ws_bytes, stream);
  if (st != FIGARO_OK) return st;
  if (R_out && ldr < c.p.n) return FIGARO_ERR_INVALID_ARG;
  const int host_out = opt && (opt->flags & FIGARO_FLAG_HOST_OUTPUT);
  return run_qr_svd(c, R_out, R_out ? ldr : c.p.n, sigma, host_out);
}

figaro_status figaro_join_svd(const figaro_table* A, const figaro_table* B, const figaro_options* opt, double* sigma,
                              double* V, int64_t ldv, double* R_out, int64_t ldr, void* ws, size_t ws_bytes,
                              void* stream) {
  if (!sigma || !V) return FIGARO_ERR_INVALID_ARG;
  if (opt && (opt->flags & (FIGARO_FLAG_HOST_OUTPUT | FIGARO_FLAG_SIGMA_DQDS))) return FIGARO_ERR_UNSUPPORTED;
  Call c;
  StageJoin join_at_exit{c};
  figaro_status st = prepare(c, A, B, opt, ws, ws_bytes, stream);
  if (st != FIGARO_OK) return st;
  if (ldv < c.p.n || (R_out && ldr < c.p.n)) return FIGARO_ERR_INVALID_ARG;
  st = run_grouping(c);
  if (st != FIGARO_OK) return st;
  st = run_factor(c, R_out, R_out ? ldr : c.p.n);
  if (st != FIGARO_OK) return st;
  FIGARO_TRY(launch_svd_v(c.p, c.p.R, c.p.n, sigma, V, ldv, c.s));
  FIGARO_TRY(c.mark(8));
  return FIGARO_OK;
}

figaro_status figaro_join_least_squares(const figaro_table* A, const figaro_table* B, const figaro_options* opt,
                                        double* beta, double* residual, void* ws, size_t ws_bytes, void* stream) {
  if (!beta || !residual) return FIGARO_ERR_INVALID_ARG;
  Call c;
  StageJoin join_at_exit{c};
  figaro_status st = prepare(c, A, B, opt, ws, ws_bytes, stream);
  if (st != FIGARO_OK) return st;
  if (c.p.n < 2) return FIGARO_ERR_INVALID_ARG;  // at least one feature besides the label
  // a label that depends on the features is an exact fit, not a rank defect
  if (c.p.report_rank > c.p.n - 1) c.p.report_rank = c.p.n - 1;
  const int host_out = opt && (opt->flags & FIGARO_FLAG_HOST_OUTPUT);
  st = run_grouping(c);
  if (st != FIGARO_OK) return st;
  st = run_factor(c, nullptr, c.p.n);
  if (st != FIGARO_OK) return st;
  // host outputs go through the workspace's sigma array (n doubles: beta, then the residual)
  double* b_dev = host_out ? c.p.sigma : beta;
  double* r_dev = host_out ? c.p.sigma + (c.p.n - 1) : residual;
  FIGARO_TRY(launch_lsq(c.p, b_dev, r_dev, c.s));
  FIGARO_TRY(c.mark(8));
  if (host_out) {
    FIGARO_TRY(cudaMemcpyAsync(beta, b_dev, sizeof(double) * (c.p.n - 1), cudaMemcpyDeviceToHost, c.s));
    FIGARO_TRY(cudaMemcpyAsync(residual, r_dev, sizeof(double), cudaMemcpyDeviceToHost, c.s));
  }
  return FIGARO_OK;
}

figaro_status figaro_triangular_singular_values(const double* R, int64_t ldr, int64_t stride, int32_t n,
                                                int32_t count, double* sigma, int32_t* info, void* stream) {
  if (!R || !sigma || n < 1 || count < 0 || ldr < n || stride < 0) return FIGARO_ERR_INVALID_ARG;
  if (n > kMaxWidth) return FIGARO_ERR_UNSUPPORTED;
  if (count == 0) return FIGARO_OK;
  figaro_status st = bind_device(R);
  if (st != FIGARO_OK) return st;
  FIGARO_TRY(launch_sigma_dqds_many(R, ldr, stride, n, count, sigma, info, static_cast<cudaStream_t>(stream)));
  return FIGARO_OK;
}

figaro_status figaro_join_singular_values_fixed(const figaro_table* A, const figaro_table* B,
                                                const figaro_options* opt, double* sigma, double* R_out,
                                                int64_t ldr, void** scratch_out, void* stream) {
  if (!sigma) return FIGARO_ERR_INVALID_ARG;
  figaro_status st = check_pair(A, B, opt);
  if (st != FIGARO_OK) return st;
  st = bind_input_device(A, B);
  if (st != FIGARO_OK) return st;
  size_t need = 0;
  st = figaro_workspace_size(A, B, opt, &need);
  if (st != FIGARO_OK) return st;
  if (need > FIGARO_FIXED_SCRATCH_BYTES) return FIGARO_ERR_WORKSPACE_TOO_SMALL;
  void* ws = nullptr;
  st = fixed_scratch(&ws);
  if (st != FIGARO_OK) return st;
  if (scratch_out) *scratch_out = ws;
  return figaro_join_singular_values(A, B, opt, sigma, R_out, ldr, ws, FIGARO_FIXED_SCRATCH_BYTES, stream);
}

figaro_status figaro_batch_workspace_size(int32_t count, const figaro_table* A, const figaro_table* B,
                                          const figaro_options* opt, size_t* bytes) {
  if (count < 0 || !bytes || (count > 0 && (!A || !B))) return FIGARO_ERR_INVALID_ARG;
  size_t total = batch_area_bytes(count);
  for (int32_t i = 0; i < count; ++i) {
    size_t one = 0;
    figaro_status st = figaro_workspace_size(&A[i], &B[i], opt, &one);
    if (st != FIGARO_OK) return st;
    total += (one + 255) & ~static_cast<size_t>(255);
  }
  *bytes = total;
  return FIGARO_OK;
}

figaro_status figaro_batch_join(int32_t count, const figaro_table* A, const figaro_table* B,
                                const figaro_options* opt, double* const* R, double* const* sigma, void* ws,
                                size_t ws_bytes, void* stream) {
  if (count < 0 || (count > 0 && (!A || !B || !R || !sigma))) return FIGARO_ERR_INVALID_ARG;
  size_t need = 0;
  figaro_status st = figaro_batch_workspace_size(count, A, B, opt, &need);
  if (st != FIGARO_OK) return st;
  if (ws_bytes < need) return FIGARO_ERR_WORKSPACE_TOO_SMALL;
  char* area = static_cast<char*>(ws);
  const size_t area_bytes = batch_area_bytes(count);
  char* base = area + area_bytes;
  const int host_out = opt && (opt->flags & FIGARO_FLAG_HOST_OUTPUT);
  // instances the batched launches take: narrow widths, device-resident
  // tables and device outputs; the others run one after another
  std::vector<Call> batched;
  std::vector<BatchOut> outs;
  std::vector<int> single;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int32_t i = 0; i < count; ++i) {
    size_t one = 0;
    figaro_workspace_size(&A[i], &B[i], opt, &one);
    one = (one + 255) & ~static_cast<size_t>(255);
    figaro_options oi = resolve(opt);
    oi.phase_events = nullptr;
    Call c;
    StageJoin join_at_exit{c};
    st = prepare(c, &A[i], &B[i], &oi, base, one, stream);
    if (st != FIGARO_OK) return st;
    base += one;
    if (!R[i] && !sigma[i]) continue;
    // (the shifted CholeskyQR3's third pass and the presorted grouping run in single calls only)
    const bool narrow = c.p.n <= kMaxWidth && !c.p.shifted && !c.p.presorted;
    const bool device_io = A[i].memory == FIGARO_MEM_DEVICE && B[i].memory == FIGARO_MEM_DEVICE && !host_out;
    if (narrow && device_io) {
      batched.push_back(c);
      outs.push_back(BatchOut{R[i], sigma[i]});
    } else {
      const int n = c.p.n;
      st = run_qr_svd(c, R[i], n, sigma[i], host_out);
      if (st != FIGARO_OK) return st;
    }
  }
  if (!batched.empty()) {
    // every batched instance was prepared on the workspace's device
    st = bind_device(area);
    if (st != FIGARO_OK) return st;
    BatchSchedule sched = schedule_for(batched);
    if (opt && (opt->flags & FIGARO_FLAG_AUTOTUNE)) {
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return FIGARO_ERR_CUDA;
      if (cs == cudaStreamCaptureStatusNone) {
        const TuneKey key = tune_key(batched);
        bool have = false;
        {
          std::lock_guard<std::mutex> lock(g_tune_mu);
          have = g_tuned.count(key) != 0;
        }
        if (!have) {
          st = tune_batch(batched, outs, area, area_bytes, s, &sched);
          if (st != FIGARO_OK) return st;
          std::lock_guard<std::mutex> lock(g_tune_mu);
          g_tuned[key] = sched;
        }
      }
    }
    st = run_batched(batched, outs, area, area_bytes, s, opt ? opt->phase_events : nullptr, sched);
    if (st != FIGARO_OK) return st;
  }
  return FIGARO_OK;
}

figaro_status figaro_batch_schedule(int32_t count, const figaro_table* A, const figaro_table* B,
                                    const figaro_options* opt, int64_t* gram_rows_per_cta, int32_t* ht_ctas_per_sm) {
  if (count < 0 || (count > 0 && (!A || !B)) || !gram_rows_per_cta || !ht_ctas_per_sm) return FIGARO_ERR_INVALID_ARG;
  std::vector<Call> calls;
  for (int32_t i = 0; i < count; ++i) {
    figaro_status st = check_pair(&A[i], &B[i], opt);
    if (st != FIGARO_OK) return st;
    const figaro_options o = resolve(opt);
    Call c;
    plan_layout(c.p, nullptr, A[i].m, A[i].n, B[i].m, B[i].n, A[i].dtype == FIGARO_F64, o.path == FIGARO_PATH_MIXED,
                0, 0, sm_count());
    if (c.p.n <= kMaxWidth && !(o.flags & (FIGARO_FLAG_SHIFTED_CHOLQR3 | FIGARO_FLAG_PRESORTED))) calls.push_back(c);
  }
  const BatchSchedule sc = schedule_for(calls);
  *gram_rows_per_cta = sc.gram_rows_per_cta;
  *ht_ctas_per_sm = sc.ht_ctas_per_sm;
  return FIGARO_OK;
}

figaro_status figaro_batch_get_status(int32_t count, const figaro_table* A, const figaro_table* B,
                                     const figaro_options* opt, const void* ws, void* stream) {
  if (count < 0 || !ws || (count > 0 && (!A || !B))) return FIGARO_ERR_INVALID_ARG;
  const char* base = static_cast<const char*>(ws) + batch_area_bytes(count);
  figaro_status worst = FIGARO_OK;
  for (int32_t i = 0; i < count; ++i) {
    size_t one = 0;
    figaro_status st = figaro_workspace_size(&A[i], &B[i], opt, &one);
    if (st != FIGARO_OK) return st;
    st = figaro_get_status(base, stream);
    if (st != FIGARO_OK && worst == FIGARO_OK) worst = st;
    base += (one + 255) & ~static_cast<size_t>(255);
  }
  return worst;
}

figaro_status figaro_get_status(const void* ws, void* stream) {
  if (!ws) return FIGARO_ERR_INVALID_ARG;
  figaro_status st = bind_device(ws);
  if (st != FIGARO_OK) return st;
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return FIGARO_ERR_CUDA;
  int32_t bits = 0;
  if (cudaMemcpy(&bits, &static_cast<const DevHeader*>(ws)->status, sizeof(bits), cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return FIGARO_ERR_CUDA;
  if (bits & kStatusTimeout) return FIGARO_ERR_DEVICE_TIMEOUT;
  if (bits & kStatusUnsorted) return FIGARO_ERR_INVALID_ARG;
  if (bits & kStatusNotSpd) return FIGARO_ERR_NOT_SPD;
  if (bits & kStatusNoConvergence) return FIGARO_ERR_NO_CONVERGENCE;
  if (bits & kStatusRankDrop) return FIGARO_ERR_RANK_DEFICIENT;
  return FIGARO_OK;
}

figaro_status figaro_get_info(const void* ws, void* stream, figaro_info* info) {
  if (!ws || !info) return FIGARO_ERR_INVALID_ARG;
  figaro_status st = bind_device(ws);
  if (st != FIGARO_OK) return st;
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return FIGARO_ERR_CUDA;
  DevHeader h;
  if (cudaMemcpy(&h, ws, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return FIGARO_ERR_CUDA;
  info->num_runs_a = h.num_runs[0];
  info->num_runs_b = h.num_runs[1];
  info->num_groups = h.num_groups;
  info->reduced_rows = h.reduced_rows;
  info->jacobi_sweeps = h.jacobi_sweeps;
  info->dependent_columns = h.dep_cols;
  return FIGARO_OK;
}

const char* figaro_status_string(figaro_status s) {
  switch (s) {
    case FIGARO_OK: return "ok";
    case FIGARO_ERR_INVALID_ARG: return "invalid argument";
    case FIGARO_ERR_WORKSPACE_TOO_SMALL: return "workspace too small";
    case FIGARO_ERR_CUDA: return "CUDA error";
    case FIGARO_ERR_NOT_SPD: return "non-finite pivot in Cholesky (NaN or Inf in the input)";
    case FIGARO_ERR_NO_CONVERGENCE: return "Jacobi SVD did not converge within the sweep limit";
    case FIGARO_ERR_DEVICE_TIMEOUT: return "a bounded device-side wait gave up";
    case FIGARO_ERR_UNSUPPORTED: return "unsupported size or width";
    case FIGARO_ERR_RANK_DEFICIENT:
      return "a column was found numerically dependent (R has a zero row there): the join is rank-deficient "
             "or too ill-conditioned for this path";
  }
  return "unknown status";
}

int32_t figaro_version(void) { return 100; }

int64_t figaro_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
