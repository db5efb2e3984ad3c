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
// Work decomposition (persistent grid, one chunk of rows per ticket):
//   * the block's threads form CG column groups (V columns each) x S
//     sub-chunks of kHtRowsPerThread consecutive sorted rows;
//   * each thread gathers its rows through perm (vector loads), scans them
//     (compensated float-float sums on the mixed path), the sub-chunks are
//     combined with a warp-shuffle + shared-memory segmented scan, and the
//     chunk's carry-in comes from a decoupled look-back over earlier chunks
//     (bounded waits);
//   * a second pass over the registers writes the tail rows (and the head
//     row at each run's end).
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace figaro {
namespace {

constexpr uint32_t kAggReady = 1u, kIncReady = 2u, kHasStart = 4u;

struct HtArgs {
  const void* x;
  int64_t ld;
  int n;
  int cg;          // column groups (power of two), threads per row
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

template <typename Tin, int V>
__device__ __forceinline__ void load_row(const Tin* src, int ncols, Tin (&out)[V]) {
  if constexpr (V == 4 && sizeof(Tin) == 4) {
    if (ncols >= 4) {
      float4 q = *reinterpret_cast<const float4*>(src);
      out[0] = q.x; out[1] = q.y; out[2] = q.z; out[3] = q.w;
      return;
    }
  } else if constexpr (V == 2 && sizeof(Tin) == 8) {
    if (ncols >= 2) {
      double2 q = *reinterpret_cast<const double2*>(src);
      out[0] = q.x; out[1] = q.y;
      return;
    }
  }
#pragma unroll
  for (int v = 0; v < V; ++v) out[v] = v < ncols ? src[v] : Tin(0);
}

template <typename Tc, int V>
__device__ __forceinline__ void store_row(Tc* dst, int ncols, const Tc (&val)[V]) {
  if constexpr (V == 4 && sizeof(Tc) == 4) {
    if (ncols >= 4) {
      *reinterpret_cast<float4*>(dst) = make_float4(val[0], val[1], val[2], val[3]);
      return;
    }
  } else if constexpr (V == 2 && sizeof(Tc) == 8) {
    if (ncols >= 2) {
      *reinterpret_cast<double2*>(dst) = make_double2(val[0], val[1]);
      return;
    }
  } else if constexpr (V == 4 && sizeof(Tc) == 8) {
    if (ncols >= 4) {
      reinterpret_cast<double2*>(dst)[0] = make_double2(val[0], val[1]);
      reinterpret_cast<double2*>(dst)[1] = make_double2(val[2], val[3]);
      return;
    }
  } else if constexpr (V == 2 && sizeof(Tc) == 4) {
    if (ncols >= 2) {
      *reinterpret_cast<float2*>(dst) = make_float2(val[0], val[1]);
      return;
    }
  }
#pragma unroll
  for (int v = 0; v < V; ++v)
    if (v < ncols) dst[v] = val[v];
}

template <typename T, int V>
__device__ __forceinline__ void seg_combine(bool ef, const Acc<T> (&ev)[V], bool& lf, Acc<T> (&lv)[V]) {
  // (earlier) then (later): the later sum restarts if a run starts in it
  if (!lf) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      Acc<T> t = ev[v];
      t.add(lv[v]);
      lv[v] = t;
    }
  }
  lf = lf || ef;
}

__device__ __forceinline__ float tail_weight(float mo, int j, float) {
  // sqrt(mo * j / (j + 1)), correctly rounded sqrt of a correctly rounded quotient
  return __fsqrt_rn(__fdiv_rn(mo * static_cast<float>(j), static_cast<float>(j + 1)));
}
__device__ __forceinline__ double tail_weight(double mo, int j, double) {
  return sqrt(mo * static_cast<double>(j) / static_cast<double>(j + 1));
}
__device__ __forceinline__ float head_weight(float mo, int mg) { return __fsqrt_rn(__fdiv_rn(mo, static_cast<float>(mg))); }
__device__ __forceinline__ double head_weight(double mo, int mg) { return sqrt(mo / static_cast<double>(mg)); }
__device__ __forceinline__ float recip(float j) { return __frcp_rn(j); }
__device__ __forceinline__ double recip(double j) { return 1.0 / j; }

template <typename Tin, typename Tc, int V>
__global__ void __launch_bounds__(kHtThreads) head_tail_kernel(HtArgs a) {
  constexpr int RPT = kHtRowsPerThread;
  const int CG = a.cg;
  const int S = kHtThreads / CG;
  const int cg = threadIdx.x % CG;
  const int sc = threadIdx.x / CG;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int col0 = cg * V;
  const int ncols = a.n - col0;  // columns this thread owns (<= 0: none)
  const Tin* X = static_cast<const Tin*>(a.x);
  Tc* TL = static_cast<Tc*>(a.tail);
  Tc* HD = static_cast<Tc*>(a.head);
  // group g of the cross-group scan: warps when CG <= 32, sub-chunks otherwise
  const bool by_warp = CG <= 32;
  const int grp = by_warp ? warp : sc;
  const int ngrp = by_warp ? kHtThreads / 32 : S;

  __shared__ int s_chunk;
  __shared__ int s_need, s_stop, s_kind, s_chunk_start;
  __shared__ unsigned char s_gf[kHtThreads];
  __shared__ Acc<Tc> s_gv[kHtThreads * V];
  __shared__ double s_carry[kMaxWidth];

  for (;;) {
    if (threadIdx.x == 0) s_chunk = static_cast<int>(atomicAdd(a.ticket, 1u));
    __syncthreads();
    const int chunk = s_chunk;
    if (chunk >= a.chunks) break;
    const int64_t row0 = static_cast<int64_t>(chunk) * a.chunk_rows;
    const int64_t rbase = row0 + static_cast<int64_t>(sc) * RPT;

    // ---- gather this thread's rows --------------------------------------
    Tc x[RPT][V];
    int jl[RPT], mgr[RPT], mo[RPT], slot[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      int64_t i = rbase + r;
      jl[r] = -1;
      mgr[r] = 0;
      mo[r] = 0;
      slot[r] = -1;
#pragma unroll
      for (int v = 0; v < V; ++v) x[r][v] = Tc(0);
      if (i < a.m) {
        int32_t p = a.perm[i];
        int32_t u = a.seg[i];
        int32_t o = a.run_off[u];
        int32_t e = a.run_off[u + 1];
        jl[r] = static_cast<int>(i - o);
        mgr[r] = e - o;
        mo[r] = a.other[u];
        slot[r] = a.hdslot[u];
        if (ncols > 0) {
          Tin tmp[V];
          load_row<Tin, V>(X + static_cast<int64_t>(p) * a.ld + col0, ncols, tmp);
#pragma unroll
          for (int v = 0; v < V; ++v) x[r][v] = static_cast<Tc>(tmp[v]);
        }
      }
    }

    // ---- thread-local segmented scan -------------------------------------
    bool f = false;
    Acc<Tc> sv[V];
#pragma unroll
    for (int v = 0; v < V; ++v) sv[v].zero();
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      if (jl[r] == 0) {
        f = true;
#pragma unroll
        for (int v = 0; v < V; ++v) sv[v].zero();
      }
#pragma unroll
      for (int v = 0; v < V; ++v) sv[v].add(x[r][v]);
    }

    // ---- intra-warp scan across sub-chunks (lanes with the same cg) ------
    bool inf = f;
    Acc<Tc> inv[V];
#pragma unroll
    for (int v = 0; v < V; ++v) inv[v] = sv[v];
    if (by_warp) {
      for (int d = CG; d < 32; d <<= 1) {
        bool of = __shfl_up_sync(0xffffffffu, inf, d);
        Acc<Tc> ov[V];
#pragma unroll
        for (int v = 0; v < V; ++v) ov[v] = shfl_up_acc(inv[v], d);
        if (lane >= d) seg_combine<Tc, V>(of, ov, inf, inv);
      }
    }
    // exclusive within the warp: the inclusive value of the previous sub-chunk
    bool exf = false;
    Acc<Tc> exv[V];
#pragma unroll
    for (int v = 0; v < V; ++v) exv[v].zero();
    if (by_warp && CG < 32) {
      bool of = __shfl_up_sync(0xffffffffu, inf, CG);
      Acc<Tc> ov[V];
#pragma unroll
      for (int v = 0; v < V; ++v) ov[v] = shfl_up_acc(inv[v], CG);
      if (lane >= CG) {
        exf = of;
#pragma unroll
        for (int v = 0; v < V; ++v) exv[v] = ov[v];
      }
    }
    // group inclusive values to shared memory
    const bool group_last = by_warp ? (lane >= 32 - CG) : true;
    if (group_last) {
      s_gf[grp * CG + cg] = inf ? 1 : 0;
#pragma unroll
      for (int v = 0; v < V; ++v) s_gv[(grp * CG + cg) * V + v] = inv[v];
    }
    if (threadIdx.x == 0) s_need = (jl[0] > 0) ? 1 : 0;  // chunk starts inside a run
    __syncthreads();
    // prefix over earlier groups (sequential, at most 8 steps)
    {
      bool gf = false;
      Acc<Tc> gv[V];
#pragma unroll
      for (int v = 0; v < V; ++v) gv[v].zero();
      for (int g = 0; g < grp; ++g) {
        bool lf = s_gf[g * CG + cg] != 0;
        Acc<Tc> lv[V];
#pragma unroll
        for (int v = 0; v < V; ++v) lv[v] = s_gv[(g * CG + cg) * V + v];
        seg_combine<Tc, V>(gf, gv, lf, lv);
        gf = lf;
#pragma unroll
        for (int v = 0; v < V; ++v) gv[v] = lv[v];
      }
      // exclusive prefix of this thread within the chunk = groups before, then warp-exclusive
      seg_combine<Tc, V>(gf, gv, exf, exv);
    }
    // chunk aggregate (held by the last sub-chunk of each column group)
    bool chunk_start = false;
    {
      bool cf = 0;
      for (int g = 0; g < ngrp; ++g) cf = cf || (s_gf[g * CG] != 0);
      chunk_start = cf;
    }
    if (sc == S - 1 && ncols > 0) {
      bool af = exf;
      Acc<Tc> av[V];
#pragma unroll
      for (int v = 0; v < V; ++v) av[v] = exv[v];
      bool lf = f;
      Acc<Tc> lv[V];
#pragma unroll
      for (int v = 0; v < V; ++v) lv[v] = sv[v];
      seg_combine<Tc, V>(af, av, lf, lv);
#pragma unroll
      for (int v = 0; v < V; ++v)
        if (v < ncols) a.chunk_agg[static_cast<int64_t>(chunk) * a.n + col0 + v] = lv[v].to_double();
      __threadfence();
    }
    __syncthreads();

    // ---- publish the aggregate, then look back for the carry -------------
    const bool publish = !(a.withhold && chunk == 0);
    if (threadIdx.x == 0) {
      if (publish) st_release(&a.chunk_status[chunk], kAggReady | (chunk_start ? kHasStart : 0u));
      int stop = -1, kind = 0;
      if (s_need) {
        int j = chunk - 1;
        for (;;) {
          uint32_t st = ld_acquire(&a.chunk_status[j]);
          int64_t spins = 0;
          while (st == 0u) {
            if (++spins > a.spin_limit) break;
            __nanosleep(64);
            st = ld_acquire(&a.chunk_status[j]);
          }
          if (st == 0u) {  // gave up: record and continue with a zero carry
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
      s_stop = stop;
      s_kind = kind;
      s_chunk_start = chunk_start ? 1 : 0;
    }
    __syncthreads();
    const int need = s_need, stop = s_stop, kind = s_kind;
    if (sc == 0 && ncols > 0) {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        if (v >= ncols) continue;
        double c = 0.0;
        if (need && kind != 3) {
          const int col = col0 + v;
          c = (kind == 1) ? __ldcg(&a.chunk_agg[static_cast<int64_t>(stop) * a.n + col])
                          : __ldcg(&a.chunk_inc[static_cast<int64_t>(stop) * a.n + col]);
          for (int j = stop + 1; j < chunk; ++j) c += __ldcg(&a.chunk_agg[static_cast<int64_t>(j) * a.n + col]);
        }
        s_carry[col0 + v] = c;
      }
    }
    __syncthreads();
    if (!s_chunk_start) {  // inclusive prefix = carry + aggregate
      if (sc == S - 1 && ncols > 0) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
          if (v >= ncols) continue;
          const int64_t k = static_cast<int64_t>(chunk) * a.n + col0 + v;
          a.chunk_inc[k] = s_carry[col0 + v] + a.chunk_agg[k];
        }
        __threadfence();
      }
      __syncthreads();
      if (threadIdx.x == 0 && publish) st_release(&a.chunk_status[chunk], kAggReady | kIncReady);
    }

    // ---- second pass: tail rows and head rows ----------------------------
    Acc<Tc> run[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      run[v].zero();
      if (!exf && v < ncols) run[v].set_double(s_carry[col0 + v]);
      run[v].add(exv[v]);
    }
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const int64_t i = rbase + r;
      if (jl[r] < 0) continue;
      if (jl[r] == 0) {
#pragma unroll
        for (int v = 0; v < V; ++v) run[v].zero();
      }
      if (ncols > 0) {
        Tc out[V];
        if (mo[r] > 0 && jl[r] > 0) {
          const Tc w = tail_weight(static_cast<Tc>(mo[r]), jl[r], Tc(0));
          const Tc rj = recip(static_cast<Tc>(jl[r]));
#pragma unroll
          for (int v = 0; v < V; ++v) out[v] = w * (x[r][v] - run[v].value() * rj);
        } else {
#pragma unroll
          for (int v = 0; v < V; ++v) out[v] = Tc(0);
        }
        store_row<Tc, V>(TL + i * a.n + col0, ncols, out);
      }
#pragma unroll
      for (int v = 0; v < V; ++v) run[v].add(x[r][v]);
      if (jl[r] == mgr[r] - 1 && slot[r] >= 0) {  // last row of its run: head row
        Tc* hrow = HD + static_cast<int64_t>(slot[r]) * a.ld_head;
        if (mo[r] > 0) {
          const Tc hw = head_weight(static_cast<Tc>(mo[r]), mgr[r]);
#pragma unroll
          for (int v = 0; v < V; ++v)
            if (v < ncols) hrow[a.head_col0 + col0 + v] = hw * run[v].value();
        } else {
#pragma unroll
          for (int v = 0; v < V; ++v)
            if (v < ncols) hrow[a.head_col0 + col0 + v] = Tc(0);
          if (cg == 0)
            for (int c = 0; c < a.zero_n; ++c) hrow[a.zero_col0 + c] = Tc(0);
        }
      }
    }
    __syncthreads();
  }
}

template <typename Tin, typename Tc, int V>
cudaError_t launch_one(const HtArgs& a, int grid, cudaStream_t s) {
  head_tail_kernel<Tin, Tc, V><<<grid, kHtThreads, 0, s>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

// Column groups of V columns for a table of width n: a power of two, so that
// the sub-chunks of a warp line up (kHtThreads / cg sub-chunks per chunk).
int ht_column_groups(int n, int V) {
  int g = (n + V - 1) / V;
  int p = 1;
  while (p < g) p <<= 1;
  return p;
}

int ht_vector_width(int n, int64_t ld, const void* x, int in_f64) {
  const int v = in_f64 ? 2 : 4;
  bool ok = (n % v == 0) && (ld % v == 0) && ((reinterpret_cast<uintptr_t>(x) & 15u) == 0);
  return ok ? v : 1;
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
  a.ticket = &p.hdr->ticket[table];
  a.status = &p.hdr->status;
  a.spin_limit = p.spin_limit;
  a.withhold = p.withhold;
  const int V = ht_vector_width(T.n, T.ld, T.x, T.in_f64);
  a.cg = ht_column_groups(T.n, V);
  a.chunk_rows = (kHtThreads / a.cg) * kHtRowsPerThread;
  a.chunks = static_cast<int>((T.m + a.chunk_rows - 1) / a.chunk_rows);  // <= T.chunks (sized for V = 1)
  int grid = p.num_sms * 4;
  if (grid > a.chunks) grid = a.chunks;
  if (T.in_f64) {
    if (p.mixed) return V == 2 ? launch_one<double, float, 2>(a, grid, s) : launch_one<double, float, 1>(a, grid, s);
    return V == 2 ? launch_one<double, double, 2>(a, grid, s) : launch_one<double, double, 1>(a, grid, s);
  }
  if (p.mixed) return V == 4 ? launch_one<float, float, 4>(a, grid, s) : launch_one<float, float, 1>(a, grid, s);
  return V == 4 ? launch_one<float, double, 4>(a, grid, s) : launch_one<float, double, 1>(a, grid, s);
}

}  // namespace figaro
