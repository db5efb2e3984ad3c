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
// Work decomposition: every warp is an independent worker.  It takes a chunk
// of consecutive sorted rows by ticket; its lanes form CG column groups of 4
// columns x (32 / CG) row groups of 8 consecutive rows.  Each lane gathers its
// rows through perm, scans them (compensated float-float sums on the mixed
// path), the row groups are combined by a warp-shuffle segmented scan, and
// the carry from earlier chunks comes from a decoupled look-back (bounded
// waits; no block-wide barriers anywhere).  A second pass over the registers
// writes the tail rows and, at each run's last row, the head row.
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace figaro {
namespace {

constexpr uint32_t kAggReady = 1u, kIncReady = 2u, kHasStart = 4u;
constexpr int kV = 4;  // columns per lane

struct HtArgs {
  const void* x;
  int64_t ld;
  int n;
  int cg;          // column groups (power of two <= 32): lanes per row
  int64_t m;
  const int32_t* perm;
  const int32_t* seg;
  const int32_t* run_off;
  const int32_t* other;
  const int32_t* hdslot;
  void* tail;      // m x n, compute type, leading dimension n
  void* head;      // rows x ld_head, compute type
  int ld_head;
  int head_col0;   // first column of this table's part of a head row
  int zero_col0;   // A side: the other table's part of unmatched head rows is zeroed here
  int zero_n;
  uint32_t* chunk_status;
  double* chunk_agg;
  double* chunk_inc;
  int chunks;
  int chunk_rows;
  uint32_t* ticket;
  int32_t* status;
  int64_t spin_limit;
  int withhold;    // test-only: chunk 0 never publishes its look-back status
};

template <typename Tin, bool kVec>
__device__ __forceinline__ void load4(const Tin* src, int ncols, Tin (&out)[kV]) {
  if constexpr (kVec && sizeof(Tin) == 4) {
    if (ncols >= 4) {
      const float4 q = __ldg(reinterpret_cast<const float4*>(src));
      out[0] = q.x; out[1] = q.y; out[2] = q.z; out[3] = q.w;
      return;
    }
  } else if constexpr (kVec && sizeof(Tin) == 8) {
    if (ncols >= 4) {
      const double2 q0 = __ldg(reinterpret_cast<const double2*>(src));
      const double2 q1 = __ldg(reinterpret_cast<const double2*>(src) + 1);
      out[0] = q0.x; out[1] = q0.y; out[2] = q1.x; out[3] = q1.y;
      return;
    }
  }
#pragma unroll
  for (int v = 0; v < kV; ++v) out[v] = v < ncols ? src[v] : Tin(0);
}

template <typename Tc, bool kVec>
__device__ __forceinline__ void store4(Tc* dst, int ncols, const Tc (&val)[kV]) {
  if constexpr (kVec && sizeof(Tc) == 4) {
    if (ncols >= 4) {
      *reinterpret_cast<float4*>(dst) = make_float4(val[0], val[1], val[2], val[3]);
      return;
    }
  } else if constexpr (kVec && sizeof(Tc) == 8) {
    if (ncols >= 4) {
      reinterpret_cast<double2*>(dst)[0] = make_double2(val[0], val[1]);
      reinterpret_cast<double2*>(dst)[1] = make_double2(val[2], val[3]);
      return;
    }
  }
#pragma unroll
  for (int v = 0; v < kV; ++v)
    if (v < ncols) dst[v] = val[v];
}

template <typename T>
__device__ __forceinline__ void seg_combine(bool ef, const Acc<T> (&ev)[kV], bool& lf, Acc<T> (&lv)[kV]) {
  // (earlier) then (later): the later sum restarts if a run starts in it
  if (!lf) {
#pragma unroll
    for (int v = 0; v < kV; ++v) {
      Acc<T> t = ev[v];
      t.add(lv[v]);
      lv[v] = t;
    }
  }
  lf = lf || ef;
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

template <typename Tin, typename Tc, bool kVec>
__global__ void __launch_bounds__(kHtThreads) head_tail_kernel(HtArgs a) {
  constexpr int RPT = kHtRowsPerThread;
  const int CG = a.cg;
  const int lane = threadIdx.x & 31;
  const int cg = lane & (CG - 1);
  const int rg = lane / CG;            // row group inside the warp
  const int col0 = cg * kV;
  const int ncols = a.n - col0;        // columns this lane owns (<= 0: none)
  const int last_rg_lane0 = 32 - CG;   // first lane of the last row group
  const Tin* X = static_cast<const Tin*>(a.x);
  Tc* TL = static_cast<Tc*>(a.tail);
  Tc* HD = static_cast<Tc*>(a.head);

  for (;;) {
    int chunk = 0;
    if (lane == 0) chunk = static_cast<int>(atomicAdd(a.ticket, 1u));
    chunk = __shfl_sync(0xffffffffu, chunk, 0);
    if (chunk >= a.chunks) break;
    const int64_t row0 = static_cast<int64_t>(chunk) * a.chunk_rows;
    const int64_t rbase = row0 + static_cast<int64_t>(rg) * RPT;

    // ---- rows and their run structure ------------------------------------
    // seg of the row before my first and of the row after my last tell where
    // runs start and end; run-level data is loaded once per run.
    int32_t segs[RPT + 1];
#pragma unroll
    for (int r = 0; r <= RPT; ++r) {
      const int64_t i = rbase + r;
      segs[r] = i < a.m ? a.seg[i] : -1;
    }
    const int32_t seg_prev = (rbase > 0 && rbase - 1 < a.m) ? a.seg[rbase - 1] : -1;
    Tc x[RPT][kV];
    int jl[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const int64_t i = rbase + r;
#pragma unroll
      for (int v = 0; v < kV; ++v) x[r][v] = Tc(0);
      if (i < a.m && ncols > 0) {
        const int32_t p = a.perm[i];
        Tin tmp[kV];
        load4<Tin, kVec>(X + static_cast<int64_t>(p) * a.ld + col0, ncols, tmp);
#pragma unroll
        for (int v = 0; v < kV; ++v) x[r][v] = static_cast<Tc>(tmp[v]);
      }
    }
    // local index of each row inside its run
    {
      int j = 0;
      if (segs[0] >= 0) j = segs[0] == seg_prev ? static_cast<int>(rbase - a.run_off[segs[0]]) : 0;
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        if (r > 0) j = (segs[r] == segs[r - 1]) ? j + 1 : 0;
        jl[r] = segs[r] >= 0 ? j : -1;
      }
    }

    // ---- thread-local segmented scan -------------------------------------
    bool f = false;
    Acc<Tc> sv[kV];
#pragma unroll
    for (int v = 0; v < kV; ++v) sv[v].zero();
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      if (jl[r] == 0) {
        f = true;
#pragma unroll
        for (int v = 0; v < kV; ++v) sv[v].zero();
      }
#pragma unroll
      for (int v = 0; v < kV; ++v) sv[v].add(x[r][v]);
    }

    // ---- warp scan across row groups (lanes with the same cg) ------------
    bool inf = f;
    Acc<Tc> inv[kV];
#pragma unroll
    for (int v = 0; v < kV; ++v) inv[v] = sv[v];
    for (int d = CG; d < 32; d <<= 1) {
      const bool of = __shfl_up_sync(0xffffffffu, inf, d);
      Acc<Tc> ov[kV];
#pragma unroll
      for (int v = 0; v < kV; ++v) ov[v] = shfl_up_acc(inv[v], d);
      if (lane >= d) seg_combine<Tc>(of, ov, inf, inv);
    }
    // exclusive value of my row group (the inclusive one of the group before)
    bool exf = false;
    Acc<Tc> exv[kV];
    {
      const bool of = __shfl_up_sync(0xffffffffu, inf, CG);
#pragma unroll
      for (int v = 0; v < kV; ++v) {
        exv[v] = shfl_up_acc(inv[v], CG);
        if (lane < CG) exv[v].zero();
      }
      exf = lane >= CG ? of : false;
    }
    // chunk aggregate = inclusive value of the last row group
    const bool chunk_start = __shfl_sync(0xffffffffu, inf, last_rg_lane0);
    if (lane >= last_rg_lane0 && ncols > 0) {
#pragma unroll
      for (int v = 0; v < kV; ++v)
        if (v < ncols) a.chunk_agg[static_cast<int64_t>(chunk) * a.n + col0 + v] = inv[v].to_double();
      __threadfence();
    }
    __syncwarp();

    // ---- publish the aggregate, then look back for the carry -------------
    const bool publish = !(a.withhold && chunk == 0);
    const bool need = __shfl_sync(0xffffffffu, jl[0] > 0, 0);  // chunk starts inside a run
    int stop = -1, kind = 0;
    if (lane == 0) {
      if (publish) st_release(&a.chunk_status[chunk], kAggReady | (chunk_start ? kHasStart : 0u));
      if (need) {
        int j = chunk - 1;
        for (;;) {
          uint32_t st = ld_acquire(&a.chunk_status[j]);
          int64_t spins = 0;
          while (st == 0u) {
            if (++spins > a.spin_limit) break;
            __nanosleep(32);
            st = ld_acquire(&a.chunk_status[j]);
          }
          if (st == 0u) {  // gave up: record it and continue with a zero carry
            set_status(a.status, kStatusTimeout);
            stop = j;
            kind = 3;
            break;
          }
          if (st & kHasStart) {
            stop = j;
            kind = 1;
            break;
          }
          if (st & kIncReady) {
            stop = j;
            kind = 2;
            break;
          }
          --j;  // aggregate only: include it and keep walking
        }
      }
    }
    stop = __shfl_sync(0xffffffffu, stop, 0);
    kind = __shfl_sync(0xffffffffu, kind, 0);
    double carry[kV];
#pragma unroll
    for (int v = 0; v < kV; ++v) carry[v] = 0.0;
    if (need && kind != 3 && rg == 0 && ncols > 0) {
#pragma unroll
      for (int v = 0; v < kV; ++v) {
        if (v >= ncols) continue;
        const int col = col0 + v;
        double c = (kind == 1) ? __ldcg(&a.chunk_agg[static_cast<int64_t>(stop) * a.n + col])
                               : __ldcg(&a.chunk_inc[static_cast<int64_t>(stop) * a.n + col]);
        for (int j = stop + 1; j < chunk; ++j) c += __ldcg(&a.chunk_agg[static_cast<int64_t>(j) * a.n + col]);
        carry[v] = c;
      }
    }
#pragma unroll
    for (int v = 0; v < kV; ++v) carry[v] = __shfl_sync(0xffffffffu, carry[v], cg);  // from row group 0
    if (!chunk_start) {  // inclusive prefix = carry + aggregate
      if (lane >= last_rg_lane0 && ncols > 0) {
#pragma unroll
        for (int v = 0; v < kV; ++v)
          if (v < ncols) a.chunk_inc[static_cast<int64_t>(chunk) * a.n + col0 + v] = carry[v] + inv[v].to_double();
        __threadfence();
      }
      __syncwarp();
      if (lane == 0 && publish) st_release(&a.chunk_status[chunk], kAggReady | kIncReady);
    }

    // ---- second pass: tail rows and head rows ----------------------------
    Acc<Tc> run[kV];
#pragma unroll
    for (int v = 0; v < kV; ++v) {
      run[v].zero();
      if (!exf) run[v].set_double(carry[v]);
      run[v].add(exv[v]);
    }
    int32_t cur_seg = -2, mo = 0, slot = -1;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const int64_t i = rbase + r;
      if (jl[r] < 0) continue;
      if (segs[r] != cur_seg) {  // run-level data, once per run
        cur_seg = segs[r];
        mo = a.other[cur_seg];
        slot = a.hdslot[cur_seg];
      }
      if (jl[r] == 0) {
#pragma unroll
        for (int v = 0; v < kV; ++v) run[v].zero();
      }
      if (ncols > 0) {
        Tc out[kV];
        if (mo > 0 && jl[r] > 0) {
          const Tc w = tail_weight(static_cast<Tc>(mo), jl[r]);
          const Tc rj = recip(static_cast<Tc>(jl[r]));
#pragma unroll
          for (int v = 0; v < kV; ++v) out[v] = w * (x[r][v] - run[v].value() * rj);
        } else {
#pragma unroll
          for (int v = 0; v < kV; ++v) out[v] = Tc(0);
        }
        store4<Tc, kVec>(TL + i * a.n + col0, ncols, out);
      }
#pragma unroll
      for (int v = 0; v < kV; ++v) run[v].add(x[r][v]);
      if (segs[r + 1] != segs[r] && slot >= 0) {  // last row of its run: head row
        Tc* hrow = HD + static_cast<int64_t>(slot) * a.ld_head;
        const int mg = jl[r] + 1;
        if (mo > 0) {
          const Tc hw = head_weight(static_cast<Tc>(mo), mg);
#pragma unroll
          for (int v = 0; v < kV; ++v)
            if (v < ncols) hrow[a.head_col0 + col0 + v] = hw * run[v].value();
        } else {
#pragma unroll
          for (int v = 0; v < kV; ++v)
            if (v < ncols) hrow[a.head_col0 + col0 + v] = Tc(0);
          if (cg == 0)
            for (int c = 0; c < a.zero_n; ++c) hrow[a.zero_col0 + c] = Tc(0);
        }
      }
    }
  }
}

template <typename Tin, typename Tc, bool kVec>
cudaError_t launch_one(const HtArgs& a, int grid, cudaStream_t s) {
  head_tail_kernel<Tin, Tc, kVec><<<grid, kHtThreads, 0, s>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

// Lanes per row for a table of width n: ceil(n / 4) rounded up to a power of
// two (at most 32 for n <= 128).
int ht_column_groups(int n) {
  const int g = (n + kV - 1) / kV;
  int p = 1;
  while (p < g) p <<= 1;
  return p;
}

int ht_chunk_rows(int n) { return (32 / ht_column_groups(n)) * kHtRowsPerThread; }

static bool ht_vector_ok(int n, int64_t ld, const void* x, int in_f64) {
  const int e = in_f64 ? 8 : 4;
  return (n % kV == 0) && ((ld * e) % 16 == 0) && ((reinterpret_cast<uintptr_t>(x) & 15u) == 0);
}

cudaError_t launch_head_tail(const Plan& p, int table, cudaStream_t s) {
  const TableWork& T = p.t[table];
  if (T.m == 0 || T.chunks == 0) return cudaSuccess;
  HtArgs a;
  a.x = T.x;
  a.ld = T.ld;
  a.n = T.n;
  a.m = T.m;
  a.perm = T.perm;
  a.seg = T.seg;
  a.run_off = T.run_off;
  a.other = T.other;
  a.hdslot = T.hdslot;
  a.tail = T.tail;
  a.head = p.head;
  a.ld_head = p.n;
  a.head_col0 = table == 0 ? 0 : p.n1;
  a.zero_col0 = table == 0 ? p.n1 : 0;
  a.zero_n = table == 0 ? p.n2 : 0;
  a.chunk_status = T.chunk_status;
  a.chunk_agg = T.chunk_agg;
  a.chunk_inc = T.chunk_inc;
  a.cg = ht_column_groups(T.n);
  a.chunk_rows = ht_chunk_rows(T.n);
  a.chunks = T.chunks;
  a.ticket = &p.hdr->ticket[table];
  a.status = &p.hdr->status;
  a.spin_limit = p.spin_limit;
  a.withhold = p.withhold;
  const bool vec = ht_vector_ok(T.n, T.ld, T.x, T.in_f64);
  const int warps_per_block = kHtThreads / 32;
  int grid = p.num_sms * 8;
  const int need = (a.chunks + warps_per_block - 1) / warps_per_block;
  if (grid > need) grid = need;
  if (T.in_f64) {
    if (p.mixed) return vec ? launch_one<double, float, true>(a, grid, s) : launch_one<double, float, false>(a, grid, s);
    return vec ? launch_one<double, double, true>(a, grid, s) : launch_one<double, double, false>(a, grid, s);
  }
  if (p.mixed) return vec ? launch_one<float, float, true>(a, grid, s) : launch_one<float, float, false>(a, grid, s);
  return vec ? launch_one<float, double, true>(a, grid, s) : launch_one<float, double, false>(a, grid, s);
}

}  // namespace figaro
