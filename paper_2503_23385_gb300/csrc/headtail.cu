// Segmented QR head / QR tail of every key group (Section 1: the H and T
// operators; Claim 1 applied per key group, then once more to the group's
// head rows, which gives the weights sqrt(m2g) on A's side and sqrt(m1g) on
// B's side).
//
// For the i-th row of a table in key order, with local index j inside its
// run (j = 0 for the run's first row), S the sum of the run's first j rows,
// mg the run length and mo the size of the partner run in the other table:
//   tail row  (j >= 1):  sqrt(mo) * sqrt(j / (j+1)) * (x - S / j)
//   head part (run end): sqrt(mo / mg) * S_total       (= sqrt(mo) * H)
// sqrt(j/(j+1)) (x - S/j) is the paper's T row (sqrt(j) x - S/sqrt(j)) /
// sqrt(j+1) written around the running mean, so that large column means do
// not cancel in FP32.
//
// Work decomposition.  The sorted rows are cut into chunks whose boundaries
// sit near multiples of L: the boundary at k L moves back to the start of
// the run containing row k L when that run has at most L rows, so a chunk
// (fewer than 2 L rows) holds whole runs, except where a run longer than L
// crosses a boundary.  Only those long-run pieces need a carry (the sum of
// the run's rows before the chunk), and it is computed before the main pass,
// in a fixed order (results are bitwise reproducible):
//   1. ht_plan:  per chunk (one warp), its first row and flags; for a chunk
//                whose end falls inside a long run, the FP64 sum of its rows
//                of that run (the "piece").
//   2. ht_scan:  per table column, a segmented scan of the pieces along each
//                long run gives every chunk's carry.
//   3. ht_stream: persistent CTAs, each streaming a contiguous range of
//                chunks tile by tile (see below): rows gathered through perm
//                with cp.async, a segmented scan per (column, row slice)
//                with compensated float-float sums on the mixed path, tail
//                rows written back contiguously, the head part at each run's
//                last row.
// With uniform keys (runs much shorter than L) steps 1-2 touch only a few
// words per chunk and step 3 reads every input row once.
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "internal.h"

namespace figaro {
namespace {

constexpr int kHtBlock = 256;
constexpr uint32_t kInside = 1u;  // chunk begins inside a run (needs a carry)
constexpr uint32_t kWhole = 2u;   // chunk lies inside one run that continues past its end

struct HtTable {
  const void* x;
  int64_t ld;
  int n;
  int64_t m;
  int vec;          // 16-byte gathers (row bytes, leading dimension and base 16-byte aligned)
  int gather;       // TMA gather4 of the rows (vec, and four rows a multiple of 128 bytes)
  const int32_t* perm;
  const int32_t* seg;
  const int32_t* run_off;
  const int32_t* other;
  const int32_t* hdslot;
  const int32_t* run_info;  // per run: first row, end row, partner run size, head slot
  void* tail;       // m x n, compute type, leading dimension n
  int head_col0;    // first column of this table's part of a head row
  int zero_col0;    // A side: the other table's part of unmatched head rows is zeroed here
  int zero_n;
  int L;
  int chunks;
  int32_t* cbeg;    // chunks + 1
  uint32_t* cflag;  // chunks
  double* piece;    // chunks x n
  double* carry;    // chunks x n
  double* gram;     // pass-1 Gram partials of the tails (null: not accumulated here): per CTA of the
                    // table n x n slots, upper triangle, a float-float pair (hi, lo) in each
};

struct HtArgs {
  HtTable t[2];
  int c0;           // chunks of table 0: block g < c0 works on table 0
  void* head;       // head_rows x ld_head, compute type
  int ld_head;
  int64_t head_rows;
  int32_t* status;
};

__host__ __device__ inline int ht_align16(int v) { return (v + 15) & ~15; }

__device__ __forceinline__ bool timed_out(const int32_t* status) {
  return (*reinterpret_cast<const volatile int32_t*>(status) & kStatusTimeout) != 0;
}

__device__ __forceinline__ int64_t clamp_idx(int64_t v, int64_t hi) { return v < 0 ? 0 : (v >= hi ? hi - 1 : v); }

// First row of chunk k and whether it begins inside a run (see above).  The
// result always lies in (k L - L, k L], so a chunk has fewer than 2 L rows
// even if the run arrays were inconsistent.
__device__ int64_t chunk_begin(const HtTable& T, int k, bool& inside) {
  inside = false;
  const int64_t i = static_cast<int64_t>(k) * T.L;
  if (k == 0) return 0;
  if (i >= T.m) return T.m;
  const int64_t r = clamp_idx(T.seg[i], T.m);
  const int64_t s = T.run_off[r], e = T.run_off[r + 1];
  if (s <= i && i < e && i - s < T.L && e - s <= T.L) return s;
  inside = s != i;
  return i;
}

template <typename Tin, typename Tc>
__device__ __forceinline__ double as_compute_double(const Tin* X, int64_t off) {
  return static_cast<double>(static_cast<Tc>(X[off]));
}

// 1. chunk table and long-run pieces: one warp per chunk
constexpr int kPlanWarps = kHtBlock / 32;
template <typename Tin, typename Tc>
__device__ __forceinline__ void ht_plan_body(const HtTable& T, const int32_t* status, int k) {
  const int lane = threadIdx.x & 31;
  if (timed_out(status)) return;
  int64_t lo = 0, hi = 0;
  if (lane == 0) {
    bool in0, in1;
    const int64_t b0 = chunk_begin(T, k, in0);
    const int64_t b1 = chunk_begin(T, k + 1, in1);
    uint32_t f = in0 ? kInside : 0u;
    if (in1 && b1 < T.m) {  // this chunk ends inside a long run: its piece of that run
      const int64_t r1 = clamp_idx(T.seg[b1], T.m);
      const int64_t s1 = T.run_off[r1];
      lo = s1 > b0 ? s1 : b0;
      hi = b1 < lo ? lo : b1;
      if (in0 && clamp_idx(T.seg[b0], T.m) == r1) f |= kWhole;
    }
    T.cbeg[k] = static_cast<int32_t>(b0);
    T.cflag[k] = f;
    if (k == T.chunks - 1) T.cbeg[T.chunks] = static_cast<int32_t>(T.m);
  }
  lo = __shfl_sync(0xffffffffu, lo, 0);
  hi = __shfl_sync(0xffffffffu, hi, 0);
  if (hi <= lo) return;
  // lanes own columns lane, lane + 32, ...; rows in order (fixed summation
  // order).  FP32 compute type: float-float sums (FP64 adds are slow on this
  // GPU); FP64 compute type: FP64 sums.
  const Tin* X = static_cast<const Tin*>(T.x);
  const int n = T.n;
  for (int c0 = 0; c0 < n; c0 += 32) {
    const int c = c0 + lane;
    double sum = 0.0;
    int64_t i = lo;
    if constexpr (sizeof(Tc) == 4) {
      float h0 = 0.f, l0 = 0.f;
      auto add = [&](float v) {
        float s_, e_;
        two_sum(h0, v, s_, e_);
        h0 = s_;
        l0 = __fadd_rn(l0, e_);
      };
      for (; i + 4 <= hi; i += 4) {
        int32_t row[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) row[u] = static_cast<int32_t>(clamp_idx(T.perm[i + u], T.m));
        float v[4] = {0.f, 0.f, 0.f, 0.f};
        if (c < n) {
#pragma unroll
          for (int u = 0; u < 4; ++u) v[u] = static_cast<float>(X[row[u] * T.ld + c]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) add(v[u]);
      }
      for (; i < hi; ++i) {
        const int64_t row = clamp_idx(T.perm[i], T.m);
        if (c < n) add(static_cast<float>(X[row * T.ld + c]));
      }
      sum = static_cast<double>(h0) + static_cast<double>(l0);
    } else {
      for (; i + 4 <= hi; i += 4) {
        int64_t row[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) row[u] = clamp_idx(T.perm[i + u], T.m);
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        if (c < n) {
#pragma unroll
          for (int u = 0; u < 4; ++u) v[u] = as_compute_double<Tin, Tc>(X, row[u] * T.ld + c);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) sum += v[u];
      }
      for (; i < hi; ++i) {
        const int64_t row = clamp_idx(T.perm[i], T.m);
        if (c < n) sum += as_compute_double<Tin, Tc>(X, row * T.ld + c);
      }
    }
    if (c < n) T.piece[static_cast<int64_t>(k) * n + c] = sum;
  }
}

template <typename Tin, typename Tc>
__global__ void __launch_bounds__(kHtBlock, 8) ht_plan_kernel(HtArgs a, int total) {  // 8 CTAs per SM: latency-bound
  pdl_enter();
  const int g = blockIdx.x * kPlanWarps + (threadIdx.x >> 5);
  if (g >= total) return;
  const int t = g < a.c0 ? 0 : 1;
  ht_plan_body<Tin, Tc>(a.t[t], a.status, t ? g - a.c0 : g);
}

// 2. carries: per (table, column), I_q = piece_q + (whole_q ? I_{q-1} : 0)
// and carry_k = I_{k-1} for every chunk k that begins inside a run.  Thread
// t of the CTA owns a contiguous range of chunks; its loads are issued in
// batches of kScanBatch (flags and pieces both, the piece selected by the
// flag afterwards) so that a range costs a few memory round trips; the
// ranges' aggregates are combined by a segmented Hillis-Steele scan in
// shared memory (log2 NT steps), then each thread walks its range again
// from its carry-in and writes the carries.  A first look at the flags alone
// ends the kernel when no chunk begins inside a run.
constexpr int kScanBatch = 8;
constexpr int kScanWide = 1024;  // threads per column when a table has many chunks
template <int NT>
__device__ __forceinline__ void ht_scan_body(const HtTable& T, const int32_t* status, int c) {
  __shared__ double s_agg[NT];
  __shared__ int s_head[NT];
  __shared__ int s_skip;
  const int K = T.chunks;
  const int t = static_cast<int>(threadIdx.x);
  if (t == 0) s_skip = (K == 0 || timed_out(status)) ? 1 : 0;
  __syncthreads();
  if (s_skip) return;
  const int n = T.n;
  const int per = (K + NT - 1) / NT;
  const int q0 = t * per < K ? t * per : K, q1 = q0 + per < K ? q0 + per : K;
  // nothing to do unless a chunk begins inside a run (uniform keys: no run is longer than L);
  // the flags alone decide it, before any piece is read
  {
    uint32_t in = 0u;
    for (int qb = q0; qb < q1; qb += kScanBatch) {
#pragma unroll
      for (int u = 1; u <= kScanBatch; ++u) in |= (qb + u <= q1 && qb + u < K) ? T.cflag[qb + u] : 0u;
    }
    if (!__syncthreads_or((in & kInside) != 0u)) return;
  }
  // flags f[u] of chunks qb + u (u <= kScanBatch: the next chunk's kInside
  // bit decides whether piece qb + u counts) and the pieces themselves
  uint32_t f[kScanBatch + 1];
  double p[kScanBatch];
  auto load = [&](int qb) {
#pragma unroll
    for (int u = 0; u <= kScanBatch; ++u) f[u] = qb + u < K ? T.cflag[qb + u] : 0u;
#pragma unroll
    for (int u = 0; u < kScanBatch; ++u) p[u] = qb + u < q1 ? T.piece[static_cast<int64_t>(qb + u) * n + c] : 0.0;
  };
  double agg = 0.0;
  int head = 0;
  for (int qb = q0; qb < q1; qb += kScanBatch) {
    load(qb);
#pragma unroll
    for (int u = 0; u < kScanBatch; ++u) {
      if (qb + u < q1) {
        if (!(f[u] & kWhole)) {
          agg = 0.0;
          head = 1;
        }
        agg += (f[u + 1] & kInside) ? p[u] : 0.0;  // (an unused piece may be unset: selected, never added)
      }
    }
  }
  // inclusive segmented scan of the ranges' (aggregate, head) pairs
  s_agg[t] = agg;
  s_head[t] = head;
  __syncthreads();
  for (int d = 1; d < NT; d <<= 1) {
    double a2 = 0.0;
    int h2 = 0;
    if (t >= d) {
      a2 = s_agg[t - d];
      h2 = s_head[t - d];
    }
    __syncthreads();
    if (t >= d) {
      if (!head) agg = a2 + agg;
      head |= h2;
      s_agg[t] = agg;
      s_head[t] = head;
    }
    __syncthreads();
  }
  double I = t > 0 ? s_agg[t - 1] : 0.0;
  for (int qb = q0; qb < q1; qb += kScanBatch) {
    load(qb);
#pragma unroll
    for (int u = 0; u < kScanBatch; ++u) {
      if (qb + u < q1) {
        const bool next_inside = (f[u + 1] & kInside) != 0;
        I = ((f[u] & kWhole) ? I : 0.0) + (next_inside ? p[u] : 0.0);
        if (next_inside) T.carry[static_cast<int64_t>(qb + u + 1) * n + c] = I;
      }
    }
  }
}

template <int NT>
__global__ void __launch_bounds__(NT) ht_scan_kernel(HtArgs a, int n0) {
  pdl_enter();
  const int t = static_cast<int>(blockIdx.x) < n0 ? 0 : 1;
  ht_scan_body<NT>(a.t[t], a.status, t ? blockIdx.x - n0 : blockIdx.x);
}

__device__ __forceinline__ float tail_weight(float mo, int j) {
  // sqrt(mo * j / (j + 1)), correctly rounded sqrt of a correctly rounded quotient
  return __fsqrt_rn(__fdiv_rn(mo * static_cast<float>(j), static_cast<float>(j + 1)));
}
__device__ __forceinline__ double tail_weight(double mo, int j) {
  return sqrt(mo * static_cast<double>(j) / static_cast<double>(j + 1));
}
__device__ __forceinline__ float head_weight(float mo, int mg) { return __fsqrt_rn(__fdiv_rn(mo, static_cast<float>(mg))); }
__device__ __forceinline__ double head_weight(double mo, int mg) { return sqrt(mo / static_cast<double>(mg)); }
__device__ __forceinline__ float recip(float j) { return __frcp_rn(j); }
__device__ __forceinline__ double recip(double j) { return 1.0 / j; }

__device__ __forceinline__ void cp_async(void* dst, const void* src, int bytes) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  if (bytes == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
  else if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}

// ---- 3. streaming head/tail pass ------------------------------------------
//
// Persistent CTAs; CTA b of a table owns a contiguous range of chunks and
// streams its rows in tiles of TR rows through a ring of kHtStages shared-
// memory stages.  Warp 0 is the producer: it reads perm and the run index of
// a tile's rows and issues cp.async copies of the rows (gathered through
// perm) and of their run data into the next free stage, which completes on
// that stage's "full" mbarrier (cp.async.mbarrier.arrive).  Warps 1-8 consume
// the stages in order: per-row weights; a segmented sum per (column, row
// slice); the slice's carry-in from the earlier slices and the state carried
// from the previous tile; tail rows stored straight to global memory (each
// warp writes whole row segments), head parts at run ends; then they free
// the stage ("empty" mbarrier).  All waits are bounded (spin_limit).
//
// Precision on the mixed path: the running sum S of a run is a float-float
// pair carried across slices and tiles; inside a slice (a few rows) and
// across the slices of one tile plain FP32 partial sums are added to it, so
// S / j carries an error of a few FP32 ulps of the partial sums, not of S.
constexpr int kHtStages = 3;
constexpr int kIdxRing = 3;  // tiles of perm / run index in flight ahead of the gathers
constexpr int kHtConsumers = 256;
constexpr int kHtStreamThreads = kHtConsumers + 32;

__host__ __device__ inline int ht_tile_rows(int n, int es_in) {
  int tr = 256;
  while (tr > 16 && tr * n * es_in > 16384) tr >>= 1;
  return tr;
}

struct HtStream {
  int TR, P;
  int stage_bytes;  // per stage: the rows (128-byte aligned), their run records
  int x, info;
  int w, rj, hw, hs, agg, flag, state, perm, bars, bytes;
};

__host__ __device__ inline int ht_align128(int v) { return (v + 127) & ~127; }

// Layout relative to a 128-byte aligned base (the launch adds 128 bytes of slack).
__host__ __device__ inline HtStream ht_stream_layout(int n, int es_in, int es_c) {
  HtStream L;
  L.TR = ht_tile_rows(n, es_in);
  L.P = kHtConsumers / n;
  const int TR = L.TR;
  int o = 0;
  L.x = o;
  o = ht_align128(o + TR * n * es_in);
  L.info = o;
  o = ht_align128(o + TR * 16);
  L.stage_bytes = o;
  o = kHtStages * L.stage_bytes;
  L.w = o;
  o = ht_align16(o + TR * es_c);
  L.rj = o;
  o = ht_align16(o + TR * es_c);
  L.hw = o;
  o = ht_align16(o + TR * es_c);
  L.hs = o;
  o = ht_align16(o + TR * 4);
  L.agg = o;  // slice sums (scalar path) or per-warp column-group totals (vector path)
  const int agg_elems = L.P * n > 8 * n ? L.P * n : 8 * n;
  o = ht_align16(o + agg_elems * es_c);
  L.flag = o;
  o = ht_align16(o + (L.P > 8 * n ? L.P : 8 * n) * 4);
  L.state = o;  // two buffers x n columns x (hi, lo) in the compute type
  o = ht_align16(o + 2 * n * 2 * es_c);
  L.perm = o;   // producer ring of row indices and run indices, kIdxRing tiles ahead
  o = ht_align16(o + kIdxRing * 2 * TR * 4);
  L.bars = o;
  o = ht_align16(o + 2 * kHtStages * 8);
  L.bytes = o + 128;
  return L;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* b, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
// Bounded wait that lets the hardware suspend the thread (up to ~20 us per
// try) until the phase completes, so waiting threads take no issue slots.
__device__ __forceinline__ bool mbar_wait_sleep(uint64_t* b, uint32_t parity, int64_t limit) {
  const int64_t tries = limit / 1024 + 1;
  for (int64_t i = 0; i < tries; ++i) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_addr(b)), "r"(parity), "r"(20000u)
        : "memory");
    if (ok) return true;
  }
  return false;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(b)) : "memory");
}
// Arrives on the mbarrier once all earlier cp.async copies of this thread are done.
__device__ __forceinline__ void cp_async_arrive(uint64_t* b) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(b)) : "memory");
}
// TMA gather of four rows (row indices r0..r3, all columns of the box) into
// shared memory, completing on the mbarrier's transaction count.
__device__ __forceinline__ void tma_gather4(void* dst, const CUtensorMap* map, int r0, int r1, int r2, int r3,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
// D += A B for one m16n8k8 TF32 warp MMA (A 16 x 8 row-major fragments a,
// B 8 x 8 column-major fragments b0, b1; FP32 accumulators).
__device__ __forceinline__ void mma_m16n8k8_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void consumers_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kHtConsumers) : "memory"); }

// Running sum of a run: float-float (hi, lo) on the mixed path, one double
// on the plain path; x is added exactly into the pair (TwoSum).
__device__ __forceinline__ void run_add(float& hi, float& lo, float x) {
  float s, e;
  two_sum(hi, x, s, e);
  hi = s;
  lo = __fadd_rn(lo, e);
}
__device__ __forceinline__ void run_add(double& hi, double& lo, double x) { hi += x; }

// Four consecutive elements: shared-memory input row piece, global tail row piece.
__device__ __forceinline__ void load4(const float* p, float (&v)[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void load4(const float* p, double (&v)[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void load4(const double* p, double (&v)[4]) {
  const double2 q0 = reinterpret_cast<const double2*>(p)[0], q1 = reinterpret_cast<const double2*>(p)[1];
  v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
}
__device__ __forceinline__ void load4(const double* p, float (&v)[4]) {
  const double2 q0 = reinterpret_cast<const double2*>(p)[0], q1 = reinterpret_cast<const double2*>(p)[1];
  v[0] = static_cast<float>(q0.x); v[1] = static_cast<float>(q0.y);
  v[2] = static_cast<float>(q1.x); v[3] = static_cast<float>(q1.y);
}
__device__ __forceinline__ void store4(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void store4(double* p, const double (&v)[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}

// V = 4: every consumer thread owns 4 consecutive columns (n a multiple of 4
// with n / 4 a power of two <= 32, tail rows 16-byte aligned); the sums of
// the row slices of one warp are combined by a warp-shuffle segmented scan,
// those of the 8 consumer warps through shared memory.  V = 1: one column
// per thread, any n.
template <typename Tin, typename Tc, int V>
__device__ __forceinline__ void ht_stream_body(const CUtensorMap* tm, const HtArgs& a, int t, int cb, int G,
                                               int64_t spin_limit) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  unsigned char* sm = sm_raw + ((128u - (smem_addr(sm_raw) & 127u)) & 127u);
  const HtTable& T = a.t[t];
  const int n = T.n;
  const HtStream L = ht_stream_layout(n, static_cast<int>(sizeof(Tin)), static_cast<int>(sizeof(Tc)));
  const int TR = L.TR, P = L.P;
  // chunk range of this CTA, and its rows
  const int k_lo = static_cast<int>(static_cast<int64_t>(cb) * T.chunks / G);
  const int k_hi = static_cast<int>(static_cast<int64_t>(cb + 1) * T.chunks / G);
  const int64_t R0 = T.cbeg[k_lo], R1 = T.cbeg[k_hi];
  if (!(R0 >= 0 && R1 <= T.m && R1 >= R0)) return;  // impossible for a consistent chunk table
  const bool inside = (T.cflag[k_lo] & kInside) != 0;
  const int ntiles = static_cast<int>((R1 - R0 + TR - 1) / TR);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + L.bars);
  uint64_t* empty = full + kHtStages;
  __shared__ int s_skip;
  if (threadIdx.x == 0) {
    for (int q = 0; q < kHtStages; ++q) {
      mbar_init(&full[q], T.gather ? 33 : 32);  // 32 cp.async arrivals (+ the TMA byte count)
      mbar_init(&empty[q], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_skip = timed_out(a.status) ? 1 : 0;  // an earlier step gave up: skip (one decision per CTA)
  }
  __syncthreads();
  if (s_skip) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    // Per tile u: the perm / run-index rows of tile u + 2 are copied into the
    // index ring (their own cp.async group), then, once tile u's indices have
    // landed (wait_group), the run data and the feature rows of tile u are
    // gathered into the stage, completing on its "full" barrier.
    const char* xb = static_cast<const char*>(T.x);
    const int64_t ldb = T.ld * static_cast<int64_t>(sizeof(Tin));
    const int row_bytes = n * static_cast<int>(sizeof(Tin));
    int32_t* ring = reinterpret_cast<int32_t*>(sm + L.perm);  // [kIdxRing][2][TR]
    auto fetch = [&](int u) {  // asynchronous copy of tile u's perm and run indices
      const int64_t r0 = R0 + static_cast<int64_t>(u) * TR;
      const int cnt = static_cast<int>(R1 - r0 < TR ? R1 - r0 : TR);
      int32_t* dp = ring + (u % kIdxRing) * 2 * TR;
      for (int r = lane; r < cnt; r += 32) {
        cp_async(dp + r, T.perm + r0 + r, 4);
        cp_async(dp + TR + r, T.seg + r0 + r, 4);
      }
    };
    for (int u = 0; u < 2; ++u) {  // always two groups, so that wait_group 2 below finds tile u's
      if (u < ntiles) fetch(u);
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    for (int u = 0; u < ntiles; ++u) {
      const int st = u % kHtStages;
      if (u >= kHtStages &&
          !mbar_wait_sleep(&empty[st], static_cast<uint32_t>(((u / kHtStages) - 1) & 1), spin_limit)) {
        set_status(a.status, kStatusTimeout);
        break;
      }
      if (u + 2 < ntiles) fetch(u + 2);
      asm volatile("cp.async.commit_group;\n" ::: "memory");  // (possibly empty) group of tile u + 2
      asm volatile("cp.async.wait_group 2;\n" ::: "memory");  // tile u's indices have landed
      __syncwarp();
      const int32_t* perm_s = ring + (u % kIdxRing) * 2 * TR;
      const int32_t* seg_s = perm_s + TR;
      unsigned char* sb = sm + st * L.stage_bytes;
      const int64_t r0 = R0 + static_cast<int64_t>(u) * TR;
      const int cnt = static_cast<int>(R1 - r0 < TR ? R1 - r0 : TR);
      if (T.gather && lane == 0) expect_tx(&full[st], static_cast<uint32_t>((cnt + 3) / 4 * 4 * row_bytes));
      __syncwarp();
      for (int r = lane; r < cnt; r += 32)  // the run record of each row
        cp_async(sb + L.info + r * 16, T.run_info + clamp_idx(seg_s[r], T.m) * 4, 16);
      if (T.gather) {
        // the rows, four per TMA gather (a short last group repeats its last row)
        for (int g4 = lane; g4 * 4 < cnt; g4 += 32) {
          int rr[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int r = g4 * 4 + q < cnt ? g4 * 4 + q : cnt - 1;
            rr[q] = static_cast<int>(clamp_idx(perm_s[r], T.m));
          }
          tma_gather4(sb + L.x + g4 * 4 * row_bytes, tm, rr[0], rr[1], rr[2], rr[3], &full[st]);
        }
      } else if (T.vec) {
        // consecutive lanes copy consecutive 16-byte pieces of the stage
        const int sp = row_bytes / 16;
        for (int idx = lane; idx < cnt * sp; idx += 32) {
          const int r = idx / sp, q16 = idx - r * sp;
          cp_async(sb + L.x + idx * 16, xb + clamp_idx(perm_s[r], T.m) * ldb + q16 * 16, 16);
        }
      } else {
        for (int idx = lane; idx < cnt * n; idx += 32) {
          const int r = idx / n, c = idx - r * n;
          cp_async(sb + L.x + idx * static_cast<int>(sizeof(Tin)),
                   xb + clamp_idx(perm_s[r], T.m) * ldb + c * static_cast<int64_t>(sizeof(Tin)),
                   static_cast<int>(sizeof(Tin)));
        }
      }
      cp_async_arrive(&full[st]);
      __syncwarp();  // the index ring slot of tile u is refilled at iteration u + 1
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    return;
  }

  // -------------------------------------------------------------- consumers
  const int ct = threadIdx.x - 32;
  Tc* w_s = reinterpret_cast<Tc*>(sm + L.w);
  Tc* rj_s = reinterpret_cast<Tc*>(sm + L.rj);
  Tc* hw_s = reinterpret_cast<Tc*>(sm + L.hw);
  int32_t* hs_s = reinterpret_cast<int32_t*>(sm + L.hs);
  Tc* agg_s = reinterpret_cast<Tc*>(sm + L.agg);
  int32_t* flag_s = reinterpret_cast<int32_t*>(sm + L.flag);
  Tc* state = reinterpret_cast<Tc*>(sm + L.state);  // [2][n][2]
  const int c = ct % n, p = ct / n;
  if (ct < n) {  // carried state entering the first tile
    Acc<Tc> s0;
    s0.zero();
    if (inside) s0.set_double(T.carry[static_cast<int64_t>(k_lo) * n + ct]);
    Tc hi, lo;
    if constexpr (sizeof(Tc) == 4) {
      hi = s0.hi;
      lo = s0.lo;
    } else {
      hi = s0.v;
      lo = 0.0;
    }
    state[ct * 2] = hi;
    state[ct * 2 + 1] = lo;
  }
  Tc* HD = static_cast<Tc*>(a.head);
  Tc* TL = static_cast<Tc*>(T.tail);
  // Pass 1 of the Gram of this table's tails, when T.gram is set (FP32, 8
  // or 16 columns): after a tile's tails are written they also replace its
  // rows in the stage, and every consumer warp adds T_k^T T_k of its 8-row
  // steps k of the tile in 3 x TF32 (hi x hi + hi x lo + lo x hi) with warp
  // MMAs (m16n8k8; the A and B fragments of T^T T are the same four values
  // per lane), accumulating its 16 x 16 partial in FP32 over the CTA's
  // tiles (as D = H^T H + (2L)^T H, whose symmetric part is the Gram: two MMAs
  // per 8-column block instead of three).  The stage is released after the
  // next tile's first barrier, when every thread is past it.
  constexpr bool kGramOk = V == 4 && sizeof(Tin) == 4 && sizeof(Tc) == 4;
  const bool fuse = kGramOk && T.gram != nullptr;
  float gd0[4] = {0.f, 0.f, 0.f, 0.f}, gd1[4] = {0.f, 0.f, 0.f, 0.f};  // G[:, 0:8], G[:, 8:16] fragments
  __shared__ int s_failed;
  if (ct == 0) s_failed = 0;
  for (int u = 0; u < ntiles; ++u) {
    const int st = u % kHtStages;
    // one thread waits for the stage (suspended in hardware), the others at the named barrier
    if (ct == 0 && !mbar_wait_sleep(&full[st], static_cast<uint32_t>((u / kHtStages) & 1), spin_limit)) {
      set_status(a.status, kStatusTimeout);
      s_failed = 1;
    }
    consumers_sync();
    if (s_failed) break;
    if (fuse && u > 0 && ct == 0) mbar_arrive(&empty[(u - 1) % kHtStages]);  // tile u - 1's Gram rows are read
    const unsigned char* sb = sm + st * L.stage_bytes;
    const Tin* xs = reinterpret_cast<const Tin*>(sb + L.x);
    const int64_t r0 = R0 + static_cast<int64_t>(u) * TR;
    const int cnt = static_cast<int>(R1 - r0 < TR ? R1 - r0 : TR);

    // per-row weights and head slots; rj = 0 marks the first row of a run
    for (int r = ct; r < cnt; r += kHtConsumers) {
      const int64_t i = r0 + r;
      const int4 info = reinterpret_cast<const int4*>(sb + L.info)[r];
      const int64_t ro = info.x, re = info.y;
      const int32_t mo = info.z;
      const int j = static_cast<int>(i - ro);
      w_s[r] = (mo > 0 && j > 0) ? tail_weight(static_cast<Tc>(mo), j) : Tc(0);
      rj_s[r] = j > 0 ? recip(static_cast<Tc>(j)) : Tc(0);
      int32_t slot = -1;
      Tc hw = Tc(0);
      if (i + 1 == re) {
        slot = info.w;
        if (slot >= a.head_rows) slot = -1;
        if (mo > 0) hw = head_weight(static_cast<Tc>(mo), j + 1);
      }
      hs_s[r] = slot;
      hw_s[r] = hw;
    }
    consumers_sync();

    if constexpr (V == 4) {
      const int CG = n >> 2;  // column groups of 4, a power of two <= 32
      const int PV = kHtConsumers / CG;
      const int cg = ct & (CG - 1), pv = ct / CG;
      const int lane = ct & 31, wc = ct >> 5;
      int per = (cnt + PV - 1) / PV;
      per |= 1;  // odd slice length: the slices of a quarter warp start in different banks
      const int q0 = pv * per < cnt ? pv * per : cnt;
      const int q1 = q0 + per < cnt ? q0 + per : cnt;
      const Tin* xrow = xs + cg * 4;
      // pass 1: the slice's sums since its last run start
      Tc ai[4] = {Tc(0), Tc(0), Tc(0), Tc(0)};
      int fi = 0;
      for (int r = q0; r < q1; ++r) {
        if (rj_s[r] == Tc(0)) {
#pragma unroll
          for (int k = 0; k < 4; ++k) ai[k] = Tc(0);
          fi = 1;
        }
        Tc xv[4];
        load4(xrow + r * n, xv);
#pragma unroll
        for (int k = 0; k < 4; ++k) ai[k] += xv[k];
      }
      // inclusive segmented scan over the warp's slices of this column group
      for (int d = CG; d < 32; d <<= 1) {
        const int of = __shfl_up_sync(0xffffffffu, fi, d);
        Tc oa[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) oa[k] = __shfl_up_sync(0xffffffffu, ai[k], d);
        if (lane >= d) {
          if (!fi) {
#pragma unroll
            for (int k = 0; k < 4; ++k) ai[k] = oa[k] + ai[k];
          }
          fi |= of;
        }
      }
      int ef = __shfl_up_sync(0xffffffffu, fi, CG);
      Tc ea[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) ea[k] = __shfl_up_sync(0xffffffffu, ai[k], CG);
      if (lane < CG) {
        ef = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) ea[k] = Tc(0);
      }
      if (lane >= 32 - CG) {  // the warp's totals per column group
#pragma unroll
        for (int k = 0; k < 4; ++k) agg_s[(wc * CG + cg) * 4 + k] = ai[k];
        flag_s[wc * CG + cg] = fi;
      }
      consumers_sync();
      // carry from the earlier warps, then from the previous tile
      int v0 = wc - 1;
      while (v0 >= 0 && !flag_s[v0 * CG + cg]) --v0;
      Tc hi[4], lo[4], loc[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        hi[k] = Tc(0);
        lo[k] = Tc(0);
        loc[k] = Tc(0);
      }
      if (!ef) {
        for (int v = v0 < 0 ? 0 : v0; v < wc; ++v) {
#pragma unroll
          for (int k = 0; k < 4; ++k) loc[k] += agg_s[(v * CG + cg) * 4 + k];
        }
        if (v0 < 0) {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            hi[k] = state[((u & 1) * n + cg * 4 + k) * 2];
            lo[k] = state[((u & 1) * n + cg * 4 + k) * 2 + 1];
          }
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) loc[k] += ea[k];
      // pass 2: tail rows and head parts
      for (int r = q0; r < q1; ++r) {
        const Tc rj = rj_s[r];
        if (rj == Tc(0)) {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            hi[k] = Tc(0);
            lo[k] = Tc(0);
            loc[k] = Tc(0);
          }
        }
        Tc xv[4], out[4];
        load4(xrow + r * n, xv);
        const Tc w = w_s[r];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const Tc S = hi[k] + (lo[k] + loc[k]);  // the run's sum of the rows before this one
          out[k] = w * fma(-S, rj, xv[k]);
          loc[k] += xv[k];
        }
        store4(TL + (r0 + r) * n + cg * 4, out);
        if (fuse) store4(const_cast<Tc*>(reinterpret_cast<const Tc*>(xrow)) + r * n, out);  // (this thread's own row slice)
        const int32_t slot = hs_s[r];
        if (slot >= 0) {
          Tc* hrow = HD + static_cast<int64_t>(slot) * a.ld_head;
          const Tc hw = hw_s[r];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int col = cg * 4 + k;
            if (hw > Tc(0)) {
              hrow[T.head_col0 + col] = hw * (hi[k] + (lo[k] + loc[k]));
            } else {
              hrow[T.head_col0 + col] = Tc(0);
              for (int cc = col; cc < T.zero_n; cc += n) hrow[T.zero_col0 + cc] = Tc(0);
            }
          }
        }
      }
      if (q1 == cnt && q0 < q1) {  // the slice holding the tile's last row carries the state on
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          run_add(hi[k], lo[k], loc[k]);
          state[(((u + 1) & 1) * n + cg * 4 + k) * 2] = hi[k];
          state[(((u + 1) & 1) * n + cg * 4 + k) * 2 + 1] = lo[k];
        }
      }
    } else {
      // pass 1: per (column, row slice), the sum since the slice's last run start
      int per = (cnt + P - 1) / P;
      per |= 1;  // odd slice length: slices of one warp start in different banks
      const int q0 = p * per < cnt ? p * per : cnt;
      const int q1 = q0 + per < cnt ? q0 + per : cnt;
      if (p < P) {
        Tc acc = Tc(0);
        int f = 0;
        for (int r = q0; r < q1; ++r) {
          if (rj_s[r] == Tc(0)) {
            acc = Tc(0);
            f = 1;
          }
          acc += static_cast<Tc>(xs[r * n + c]);
        }
        agg_s[p * n + c] = acc;
        if (c == 0) flag_s[p] = f;
      }
      consumers_sync();

      // pass 2: carry into the slice, tail rows, head parts
      if (p < P) {
        int v0 = p - 1;
        while (v0 >= 0 && !flag_s[v0]) --v0;
        Tc hi = Tc(0), lo = Tc(0), loc = Tc(0);
        if (v0 < 0) {
          hi = state[((u & 1) * n + c) * 2];
          lo = state[((u & 1) * n + c) * 2 + 1];
        }
        for (int v = v0 < 0 ? 0 : v0; v < p; ++v) loc += agg_s[v * n + c];
        for (int r = q0; r < q1; ++r) {
          const Tc rj = rj_s[r];
          if (rj == Tc(0)) {
            hi = Tc(0);
            lo = Tc(0);
            loc = Tc(0);
          }
          const Tc xv = static_cast<Tc>(xs[r * n + c]);
          const Tc S = hi + (lo + loc);  // the run's sum of the rows before this one
          TL[(r0 + r) * n + c] = w_s[r] * fma(-S, rj, xv);
          loc += xv;
          const int32_t slot = hs_s[r];
          if (slot >= 0) {
            Tc* hrow = HD + static_cast<int64_t>(slot) * a.ld_head;
            const Tc hw = hw_s[r];
            if (hw > Tc(0)) {
              hrow[T.head_col0 + c] = hw * (hi + (lo + loc));
            } else {
              hrow[T.head_col0 + c] = Tc(0);
              for (int cc = c; cc < T.zero_n; cc += n) hrow[T.zero_col0 + cc] = Tc(0);
            }
          }
        }
        if (q1 == cnt && q0 < q1) {  // the slice holding the tile's last row carries the state on
          run_add(hi, lo, loc);
          state[(((u + 1) & 1) * n + c) * 2] = hi;
          state[(((u + 1) & 1) * n + c) * 2 + 1] = lo;
        }
      }
    }
    consumers_sync();
    if (fuse) {
      const float* tt = reinterpret_cast<const float*>(sb + L.x);  // the tile's tails, rows of n
      const int gq = (ct & 31) >> 2, tq = ct & 3;
      const int ksteps = (cnt + 7) >> 3;
      for (int ks = ct >> 5; ks < ksteps; ks += kHtConsumers / 32) {
        const int ra = ks * 8 + tq, rb = ra + 4;
        const float v[4] = {ra < cnt ? tt[ra * n + gq] : 0.f, (n > 8 && ra < cnt) ? tt[ra * n + gq + 8] : 0.f,
                            rb < cnt ? tt[rb * n + gq] : 0.f, (n > 8 && rb < cnt) ? tt[rb * n + gq + 8] : 0.f};
        uint32_t h[4], l2[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          h[k] = __float_as_uint(v[k]) & 0xffffe000u;  // TF32 hi: truncation
          const uint32_t lo = (__float_as_uint(__fsub_rn(v[k], __uint_as_float(h[k]))) + 0x1000u) & 0xffffe000u;
          l2[k] = __float_as_uint(2.f * __uint_as_float(lo));  // 2 lo (exact): D = H^T H + (2L)^T H, G = (D + D^T) / 2
        }
        mma_m16n8k8_tf32(gd0, l2, h[0], h[2]);
        mma_m16n8k8_tf32(gd0, h, h[0], h[2]);
        if (n > 8) {
          mma_m16n8k8_tf32(gd1, l2, h[1], h[3]);
          mma_m16n8k8_tf32(gd1, h, h[1], h[3]);
        }
      }
    } else if (ct == 0) {
      mbar_arrive(&empty[st]);
    }
  }
  if (fuse && !s_failed) {
    // the row groups' sums through the stage area (every tile has been
    // consumed: no copy is in flight), then the CTA's partial
    consumers_sync();
    float* red = reinterpret_cast<float*>(sm) + (ct >> 5) * 256;  // [warp][16][16]
    const int gq = (ct & 31) >> 2, tq = ct & 3;
    red[gq * 16 + 2 * tq] = gd0[0];
    red[gq * 16 + 2 * tq + 1] = gd0[1];
    red[(gq + 8) * 16 + 2 * tq] = gd0[2];
    red[(gq + 8) * 16 + 2 * tq + 1] = gd0[3];
    red[gq * 16 + 8 + 2 * tq] = gd1[0];
    red[gq * 16 + 8 + 2 * tq + 1] = gd1[1];
    red[(gq + 8) * 16 + 8 + 2 * tq] = gd1[2];
    red[(gq + 8) * 16 + 8 + 2 * tq + 1] = gd1[3];
    consumers_sync();
    const float* all = reinterpret_cast<const float*>(sm);
    float2* part = reinterpret_cast<float2*>(T.gram + static_cast<int64_t>(cb) * n * n);
    for (int e = ct; e < n * n; e += kHtConsumers) {
      const int i = e / n, j = e - (e / n) * n;
      if (i > j) continue;  // (upper triangle)
      float hh = 0.f, ll = 0.f;
      for (int w = 0; w < kHtConsumers / 32; ++w) {
        float s_, e_;
        // (the symmetric part of D: halving is exact)
        two_sum(hh, 0.5f * all[w * 256 + i * 16 + j], s_, e_);
        hh = s_;
        ll = __fadd_rn(ll, e_);
        two_sum(hh, 0.5f * all[w * 256 + j * 16 + i], s_, e_);
        hh = s_;
        ll = __fadd_rn(ll, e_);
      }
      part[i * n + j] = make_float2(hh, ll);
    }
  }
}

template <typename Tin, typename Tc, int V>
__global__ void __launch_bounds__(kHtStreamThreads, 3)  // three CTAs per SM (shared memory allows three)
    ht_stream_kernel(const __grid_constant__ CUtensorMap tm0, const __grid_constant__ CUtensorMap tm1, HtArgs a,
                     int g0, int g1, int64_t spin_limit) {
  pdl_enter();
  const int t = static_cast<int>(blockIdx.x) < g0 ? 0 : 1;
  ht_stream_body<Tin, Tc, V>(t ? &tm1 : &tm0, a, t, t ? static_cast<int>(blockIdx.x) - g0 : static_cast<int>(blockIdx.x),
                             t ? g1 : g0, spin_limit);
}

template <typename Tin, typename Tc>
cudaError_t launch_typed_carry(const HtArgs& a, int total, int ncols, cudaStream_t s) {
  pdl_launch(ht_plan_kernel<Tin, Tc>, (total + kPlanWarps - 1) / kPlanWarps, kHtBlock, 0, s, a, total);
  const int n0 = a.t[0].chunks > 0 ? a.t[0].n : 0;
  if (a.t[0].chunks > 8 * kHtBlock || a.t[1].chunks > 8 * kHtBlock)
    pdl_launch(ht_scan_kernel<kScanWide>, ncols, kScanWide, 0, s, a, n0);
  else
    pdl_launch(ht_scan_kernel<kHtBlock>, ncols, kHtBlock, 0, s, a, n0);
  count_launches(2);
  return cudaGetLastError();
}

// Tensor map for TMA row gathers of a table: box = one full row.  Returns
// false (the caller then copies rows with cp.async) when TMA cannot address it.
bool row_gather_map(CUtensorMap* map, const HtTable& T, int es_in) {
  const int row_bytes = T.n * es_in;
  if (!T.vec || T.m < 1 || T.n > 256 || row_bytes % 32 != 0) return false;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(T.n), static_cast<cuuint64_t>(T.m)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(T.ld) * es_in};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(T.n), 1};
  cuuint32_t es[2] = {1, 1};
  const CUresult r = enc(map, es_in == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                         const_cast<void*>(T.x), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Shared memory of the stream kernel for the tables of `a` (granted above 48
// KB once per device and size) and its CTAs per SM.
template <typename Tin, typename Tc, int V>
cudaError_t ht_stream_setup(const HtArgs& a, int* smem_out, int* occ_out) {
  int smem = 0;
  for (int t = 0; t < 2; ++t)
    if (a.t[t].chunks > 0) {
      const HtStream L = ht_stream_layout(a.t[t].n, sizeof(Tin), sizeof(Tc));
      if (L.bytes > smem) smem = L.bytes;
    }
  static int granted[64] = {0};
  static int per_sm[64] = {0};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  const bool cache = dev >= 0 && dev < 64;
  if (smem > 48 * 1024 && (!cache || granted[dev] < smem)) {  // opt in to more than the default 48 KB
    err = cudaFuncSetAttribute(ht_stream_kernel<Tin, Tc, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (err != cudaSuccess) return err;
    if (cache) granted[dev] = smem;
  }
  int occ = cache ? per_sm[dev] : 0;
  if (occ <= 0) {
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ht_stream_kernel<Tin, Tc, V>, kHtStreamThreads, smem);
    if (err != cudaSuccess) return err;
    if (occ < 1) occ = 1;
    if (cache) per_sm[dev] = occ;
  }
  *smem_out = smem;
  *occ_out = occ;
  return cudaSuccess;
}

// CTAs per table in proportion to its chunks, at most one per chunk.
void ht_split(const HtArgs& a, int G, int* g0_out, int* g1_out) {
  const int c0 = a.t[0].chunks, c1 = a.t[1].chunks;
  int g0 = c0 > 0 ? static_cast<int>((static_cast<int64_t>(G) * c0 + (c0 + c1) - 1) / (c0 + c1)) : 0;
  if (c0 > 0 && g0 < 1) g0 = 1;
  if (g0 > c0) g0 = c0;
  int g1 = c1 > 0 ? G - g0 : 0;
  if (c1 > 0 && g1 < 1) g1 = 1;
  if (g1 > c1) g1 = c1;
  *g0_out = g0;
  *g1_out = g1;
}

// grid: the CTAs per table planned by ht_plan_gram1 (both 0: split here)
template <typename Tin, typename Tc, int V>
cudaError_t launch_typed_main(HtArgs a, int num_sms, const int grid[2], int64_t spin_limit, cudaStream_t s) {
  CUtensorMap maps[2];
  std::memset(maps, 0, sizeof(maps));
  for (int t = 0; t < 2; ++t)
    a.t[t].gather = a.t[t].chunks > 0 && row_gather_map(&maps[t], a.t[t], static_cast<int>(sizeof(Tin)));
  int smem = 0, occ = 0;
  const cudaError_t err = ht_stream_setup<Tin, Tc, V>(a, &smem, &occ);
  if (err != cudaSuccess) return err;
  int g0 = grid[0], g1 = grid[1];
  if (g0 + g1 == 0) ht_split(a, num_sms * occ, &g0, &g1);
  if (g0 + g1 == 0) return cudaSuccess;
  pdl_launch(ht_stream_kernel<Tin, Tc, V>, g0 + g1, kHtStreamThreads, smem, s, maps[0], maps[1], a, g0, g1, spin_limit);
  count_launches(1);
  return cudaGetLastError();
}

__host__ __device__ inline bool ht_vector_ok(int n, int64_t ld, const void* x, int in_f64) {
  const int e = in_f64 ? 8 : 4;
  return ((n * e) % 16 == 0) && ((ld * e) % 16 == 0) && ((reinterpret_cast<uintptr_t>(x) & 15u) == 0);
}

__host__ __device__ inline HtTable ht_table(const Plan& p, int t) {
  const TableWork& W = p.t[t];
  HtTable T{};
  T.x = W.x;
  T.ld = W.ld;
  T.n = W.n;
  T.m = W.m;
  T.vec = W.m > 0 && ht_vector_ok(W.n, W.ld, W.x, W.in_f64);
  T.gather = 0;
  T.perm = W.perm;
  T.seg = W.seg;
  T.run_off = W.run_off;
  T.other = W.other;
  T.hdslot = W.hdslot;
  T.run_info = W.run_info;
  T.tail = W.tail;
  T.head_col0 = t == 0 ? 0 : p.n1;
  T.zero_col0 = t == 0 ? p.n1 : 0;
  T.zero_n = t == 0 ? p.n2 : 0;
  T.L = W.chunk_rows;
  T.chunks = W.m > 0 ? W.chunks : 0;
  T.cbeg = W.cbeg;
  T.cflag = W.cflag;
  T.piece = W.piece;
  T.carry = W.carry;
  return T;
}

__host__ __device__ inline HtArgs make_args(const Plan& p) {
  HtArgs a{};
  a.t[0] = ht_table(p, 0);
  a.t[1] = ht_table(p, 1);
  a.c0 = a.t[0].chunks;
  a.head = p.head;
  a.ld_head = p.n;
  a.head_rows = p.t[0].m;
  a.status = &p.hdr->status;
  return a;
}

// 4-column consumers: a width of 4 x a power of two <= 128 and 16-byte aligned tail rows.
__host__ __device__ inline bool ht_v4_ok(const HtTable& T) {
  const int cg = T.n / 4;
  return T.n % 4 == 0 && cg >= 1 && cg <= 32 && (cg & (cg - 1)) == 0 &&
         (reinterpret_cast<uintptr_t>(T.tail) & 15u) == 0;
}

// ---- batched forms: jobs are (instance, table); aux = table
// chunk plan: first[] counts chunks, one warp per chunk
template <typename Tin, typename Tc>
__global__ void __launch_bounds__(kHtBlock) ht_plan_batched(BatchDev b, BatchJobs J, int total) {
  pdl_enter();
  const int g = blockIdx.x * kPlanWarps + (threadIdx.x >> 5);
  if (g >= total) return;
  const int j = batch_job(J, g);
  const Plan& P = b.plans[J.inst[j]];
  const HtTable T = ht_table(P, J.aux[j]);
  ht_plan_body<Tin, Tc>(T, &P.hdr->status, g - J.first[j]);
}

// carries: first[] counts columns, one CTA per column
__global__ void __launch_bounds__(kHtBlock) ht_scan_batched(BatchDev b, BatchJobs J) {
  pdl_enter();
  const int j = batch_job(J, blockIdx.x);
  const Plan& P = b.plans[J.inst[j]];
  const HtTable T = ht_table(P, J.aux[j]);
  ht_scan_body<kHtBlock>(T, &P.hdr->status, blockIdx.x - J.first[j]);
}

// streaming pass: first[] counts CTAs; rows are copied with cp.async (no TMA)
template <typename Tin, typename Tc, int V>
__global__ void __launch_bounds__(kHtStreamThreads) ht_stream_batched(BatchDev b, BatchJobs J) {
  pdl_enter();
  __shared__ HtArgs s_a;
  const int j = batch_job(J, blockIdx.x);
  const Plan& P = b.plans[J.inst[j]];
  if (threadIdx.x == 0) s_a = make_args(P);
  __syncthreads();
  ht_stream_body<Tin, Tc, V>(nullptr, s_a, J.aux[j], blockIdx.x - J.first[j], J.first[j + 1] - J.first[j],
                             P.spin_limit);
}

template <typename Tin, typename Tc>
cudaError_t launch_batch_ht_typed(const BatchDev& b, const BatchJobs& plan, int plan_total, const BatchJobs& scan,
                                  const BatchJobs* stream, const int* smem, cudaStream_t s) {
  if (plan.njobs > 0) {
    pdl_launch(ht_plan_batched<Tin, Tc>, (plan_total + kPlanWarps - 1) / kPlanWarps, kHtBlock, 0, s, b, plan, plan_total);
    pdl_launch(ht_scan_batched, scan.ctas, kHtBlock, 0, s, b, scan);
    count_launches(2);
  }
  for (int v = 0; v < 2; ++v) {
    if (stream[v].njobs == 0) continue;
    auto kern = v == 0 ? ht_stream_batched<Tin, Tc, 4> : ht_stream_batched<Tin, Tc, 1>;
    if (smem[v] > 48 * 1024) {
      cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem[v]);
      if (err != cudaSuccess) return err;
    }
    pdl_launch(kern, stream[v].ctas, kHtStreamThreads, smem[v], s, b, stream[v]);
    count_launches(1);
  }
  return cudaGetLastError();
}

}  // namespace

void ht_batch_table(const Plan& p, int t, int* variant, int* smem, int* chunks) {
  const HtTable T = ht_table(p, t);
  *chunks = T.chunks;
  *variant = ht_v4_ok(T) ? 0 : 1;
  const int ein = p.t[t].in_f64 ? 8 : 4, ec = p.mixed ? 4 : 8;
  *smem = T.chunks > 0 ? ht_stream_layout(T.n, ein, ec).bytes : 0;
}

cudaError_t launch_batch_ht(const BatchDev& b, const BatchJobs& plan, int plan_total, const BatchJobs& scan,
                            const BatchJobs stream[2], const int smem[2], int in_f64, int mixed, cudaStream_t s) {
  if (in_f64) return mixed ? launch_batch_ht_typed<double, float>(b, plan, plan_total, scan, stream, smem, s)
                           : launch_batch_ht_typed<double, double>(b, plan, plan_total, scan, stream, smem, s);
  return mixed ? launch_batch_ht_typed<float, float>(b, plan, plan_total, scan, stream, smem, s)
               : launch_batch_ht_typed<float, double>(b, plan, plan_total, scan, stream, smem, s);
}

// Chunk spacing L for a table of width n: the largest power of two in
// [16, 512] with (2 L - 1) rows of input (and output, when its type differs)
// within 32 KB of shared memory.
int ht_chunk_rows(int n, int in_f64, int mixed) {
  const int es_in = in_f64 ? 8 : 4, es_c = mixed ? 4 : 8;
  const int row = n * (es_in + (es_in != es_c ? es_c : 0));
  int L = 512;
  while (L > 16 && (2 * L - 1) * row > 32 * 1024) L >>= 1;
  return L;
}

// Arguments of the head/tail step restricted to table `only` (-1: both).
static HtArgs args_for(const Plan& p, int only) {
  HtArgs a = make_args(p);
  if (only >= 0) {
    a.t[1 - only].chunks = 0;
    a.c0 = a.t[0].chunks;
  }
  return a;
}

cudaError_t launch_ht_carry(const Plan& p, cudaStream_t s, int only) {
  const HtArgs a = args_for(p, only);
  const int grid = a.t[0].chunks + a.t[1].chunks;
  if (grid == 0) return cudaSuccess;
  const int ncols = (a.t[0].chunks > 0 ? a.t[0].n : 0) + (a.t[1].chunks > 0 ? a.t[1].n : 0);
  const bool in64 = p.t[0].in_f64 != 0;
  if (in64) return p.mixed ? launch_typed_carry<double, float>(a, grid, ncols, s)
                           : launch_typed_carry<double, double>(a, grid, ncols, s);
  return p.mixed ? launch_typed_carry<float, float>(a, grid, ncols, s)
                 : launch_typed_carry<float, double>(a, grid, ncols, s);
}

// The 4-column path needs both tables' widths to be 4 x a power of two <=
// 128 and 16-byte aligned tail rows.
static bool ht_use_v4(const HtArgs& a) {
  bool v4 = true;
  for (int t = 0; t < 2; ++t)
    if (a.t[t].chunks > 0) v4 = v4 && ht_v4_ok(a.t[t]);
  return v4;
}

cudaError_t launch_ht_main(const Plan& p, cudaStream_t s, int only) {
  HtArgs a = args_for(p, only);
  const int grid = a.t[0].chunks + a.t[1].chunks;
  if (grid == 0) return cudaSuccess;
  const bool in64 = p.t[0].in_f64 != 0;
  const int sms = p.num_sms;
  const int64_t sl = p.spin_limit;
  const bool v4 = ht_use_v4(a);
  int g[2] = {p.ht_grid[0], p.ht_grid[1]};
  if (only >= 0) g[1 - only] = 0;
  if (p.ht_gram[0] > 0 || p.ht_gram[1] > 0) {  // (planned for the FP32 4-column kernel only)
    if (in64 || !p.mixed || !v4) return cudaErrorInvalidValue;
    for (int t = 0; t < 2; ++t) a.t[t].gram = p.ht_gram[t] > 0 && a.t[t].chunks > 0 ? p.gpart[1 + t] : nullptr;
  }
  if (in64) {
    if (p.mixed) return v4 ? launch_typed_main<double, float, 4>(a, sms, g, sl, s) : launch_typed_main<double, float, 1>(a, sms, g, sl, s);
    return v4 ? launch_typed_main<double, double, 4>(a, sms, g, sl, s) : launch_typed_main<double, double, 1>(a, sms, g, sl, s);
  }
  if (p.mixed) return v4 ? launch_typed_main<float, float, 4>(a, sms, g, sl, s) : launch_typed_main<float, float, 1>(a, sms, g, sl, s);
  return v4 ? launch_typed_main<float, double, 4>(a, sms, g, sl, s) : launch_typed_main<float, double, 1>(a, sms, g, sl, s);
}

void ht_plan_gram1(Plan& p) {
  p.ht_grid[0] = p.ht_grid[1] = 0;
  p.ht_gram[0] = p.ht_gram[1] = 0;
  if (!p.mixed || p.t[0].in_f64 || p.gram_engine != 0 || p.wide) return;  // (0: the automatic engine)
  const HtArgs a = make_args(p);
  if (a.t[0].chunks + a.t[1].chunks == 0 || !ht_use_v4(a)) return;
  bool any = false;
  for (int t = 0; t < 2; ++t) {
    const int n = a.t[t].n;
    any = any || (a.t[t].chunks > 0 && (n == 8 || n == 16));
  }
  if (!any) return;
  int smem = 0, occ = 0;
  if (ht_stream_setup<float, float, 4>(a, &smem, &occ) != cudaSuccess) return;
  int g[2] = {0, 0};
  if (p.ht_split) {  // one launch per table, each on the whole GPU
    for (int t = 0; t < 2; ++t) {
      int g0 = 0, g1 = 0;
      ht_split(args_for(p, t), p.num_sms * occ, &g0, &g1);
      g[t] = t ? g1 : g0;
    }
  } else {
    ht_split(a, p.num_sms * occ, &g[0], &g[1]);
  }
  for (int t = 0; t < 2; ++t) {
    const int n = a.t[t].n;
    if (a.t[t].chunks > 0 && (n == 8 || n == 16) && p.gpart[1 + t] &&
        static_cast<int64_t>(g[t]) * n * n <= p.gcap[1 + t])
      p.ht_gram[t] = g[t];
  }
  if (p.ht_gram[0] > 0 || p.ht_gram[1] > 0) {
    p.ht_grid[0] = g[0];
    p.ht_grid[1] = g[1];
  }
}

}  // namespace figaro
