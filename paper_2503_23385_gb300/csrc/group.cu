// Key grouping of both tables: a stable LSD radix sort of (key, row index),
// run-length encoding of the sorted keys, and the matching of runs between
// the tables (the inner natural join keeps only keys present in both).
//
// The paper assumes inputs already sorted by the join attribute (Section 2,
// experimental setup); this step produces that order.  Stability keeps rows
// with equal keys in input order, which fixes the order of the QR tail rows
// inside each key group.
//
// Each launch covers both tables: blocks [0, nbA) work on A, the rest on B.
#include "common.cuh"
#include "internal.h"

namespace figaro {
namespace {

struct TwoTables {
  TableWork t[2];
  DevHeader* h;
  int nb0;  // blocks belonging to table 0
};

__device__ __forceinline__ int table_of_block(const TwoTables& a, int& local) {
  int b = blockIdx.x;
  if (b < a.nb0) {
    local = b;
    return 0;
  }
  local = b - a.nb0;
  return 1;
}

__device__ __forceinline__ int num_passes(const DevHeader* h, int t) {
  uint32_t r = h->kmax[t] - h->kmin[t];
  int bits = r ? 32 - __clz(r) : 0;
  int p = (bits + kRadixBits - 1) / kRadixBits;
  return p < 1 ? 1 : p;
}

__global__ void reset_kernel(DevHeader* h, uint32_t* s0, int n0, uint32_t* s1, int n1) {
  int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid == 0) {
    h->status = 0;
    for (int i = 0; i < 8; ++i) h->ticket[i] = 0;
    h->kmin[0] = h->kmin[1] = 0xffffffffu;
    h->kmax[0] = h->kmax[1] = 0u;
    h->num_runs[0] = h->num_runs[1] = 0;
    h->num_groups = 0;
    h->reduced_rows = 0;
    h->jacobi_sweeps = 0;
  }
  for (int i = tid; i < n0; i += gridDim.x * blockDim.x) s0[i] = 0u;
  for (int i = tid; i < n1; i += gridDim.x * blockDim.x) s1[i] = 0u;
}

__global__ void __launch_bounds__(kSortThreads) key_range_kernel(TwoTables a) {
  int tile;
  int t = table_of_block(a, tile);
  const TableWork& T = a.t[t];
  uint32_t lo = 0xffffffffu, hi = 0u;
  int64_t base = static_cast<int64_t>(tile) * kSortTile;
  for (int it = 0; it < kSortItems; ++it) {
    int64_t i = base + it * kSortThreads + threadIdx.x;
    if (i < T.m) {
      uint32_t u = key_to_ordered(T.key[i]);
      lo = min(lo, u);
      hi = max(hi, u);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&a.h->kmin[t], lo);
    atomicMax(&a.h->kmax[t], hi);
  }
}

__device__ __forceinline__ uint32_t load_sort_key(const TableWork& T, const DevHeader* h, int t, int pass,
                                                  int64_t i) {
  if (pass == 0) return key_to_ordered(T.key[i]) - h->kmin[t];
  return T.kb[(pass - 1) & 1][i];
}

__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(TwoTables a, int pass) {
  int tile;
  int t = table_of_block(a, tile);
  const TableWork& T = a.t[t];
  if (pass >= num_passes(a.h, t)) return;
  __shared__ uint32_t hist[kRadixBins];
  for (int d = threadIdx.x; d < kRadixBins; d += blockDim.x) hist[d] = 0u;
  __syncthreads();
  int64_t base = static_cast<int64_t>(tile) * kSortTile;
  int shift = pass * kRadixBits;
  for (int it = 0; it < kSortItems; ++it) {
    int64_t i = base + it * kSortThreads + threadIdx.x;
    if (i < T.m) {
      uint32_t d = (load_sort_key(T, a.h, t, pass, i) >> shift) & (kRadixBins - 1);
      atomicAdd(&hist[d], 1u);
    }
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRadixBins; d += blockDim.x)
    T.hist[static_cast<int64_t>(d) * T.tiles + tile] = hist[d];
}

// Exclusive scan of one table's digit-major histogram (bins x tiles), in place.
constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads) radix_scan_kernel(TwoTables a, int pass) {
  int t = blockIdx.x;
  const TableWork& T = a.t[t];
  if (T.m == 0 || pass >= num_passes(a.h, t)) return;
  int64_t N = static_cast<int64_t>(kRadixBins) * T.tiles;
  int64_t per = (N + kScanThreads - 1) / kScanThreads;
  int64_t lo = per * threadIdx.x;
  int64_t hi = lo + per < N ? lo + per : N;
  uint32_t sum = 0;
  for (int64_t i = lo; i < hi; ++i) sum += T.hist[i];
  // block exclusive scan of the per-thread sums
  __shared__ uint32_t wsum[32];
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = sum;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = wsum[lane];
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    wsum[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  uint32_t run = incl - sum + (warp > 0 ? wsum[warp - 1] : 0u);
  for (int64_t i = lo; i < hi; ++i) {
    uint32_t v = T.hist[i];
    T.hist[i] = run;
    run += v;
  }
}

// Stable scatter of one radix pass.  Keys of a tile are ranked in input
// order: warp w owns keys [w*512, w*512+512) of the tile, visited in 16
// rounds of 32 consecutive keys; __match_any_sync groups equal digits.
__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(TwoTables a, int pass) {
  int tile;
  int t = table_of_block(a, tile);
  const TableWork& T = a.t[t];
  if (pass >= num_passes(a.h, t)) return;
  constexpr int kWarps = kSortThreads / 32;
  __shared__ uint32_t cnt[kWarps][kRadixBins];
  __shared__ uint32_t sbase[kRadixBins];
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kWarps * kRadixBins; i += blockDim.x) (&cnt[0][0])[i] = 0u;
  for (int d = threadIdx.x; d < kRadixBins; d += blockDim.x)
    sbase[d] = T.hist[static_cast<int64_t>(d) * T.tiles + tile];
  __syncthreads();
  int shift = pass * kRadixBits;
  int64_t base = static_cast<int64_t>(tile) * kSortTile + warp * (32 * kSortItems);
  uint32_t key[kSortItems];
  int32_t val[kSortItems];
  uint32_t rank[kSortItems];
  const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    int64_t i = base + r * 32 + lane;
    bool valid = i < T.m;
    uint32_t u = 0;
    int32_t v = 0;
    if (valid) {
      u = load_sort_key(T, a.h, t, pass, i);
      v = pass == 0 ? static_cast<int32_t>(i) : T.vb[(pass - 1) & 1][i];
    }
    key[r] = u;
    val[r] = v;
    uint32_t d = valid ? ((u >> shift) & (kRadixBins - 1)) : kRadixBins;  // sentinel bin for padding
    uint32_t peers = __match_any_sync(0xffffffffu, d);
    uint32_t before = 0;
    if (valid) before = cnt[warp][d];
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) cnt[warp][d] = before + __popc(peers);
    __syncwarp();
    rank[r] = before + __popc(peers & lt_mask);
  }
  __syncthreads();
  // exclusive prefix over warps, per digit
  for (int d = threadIdx.x; d < kRadixBins; d += blockDim.x) {
    uint32_t run = 0;
    for (int w = 0; w < kWarps; ++w) {
      uint32_t c = cnt[w][d];
      cnt[w][d] = run;
      run += c;
    }
  }
  __syncthreads();
  uint32_t* ko = T.kb[pass & 1];
  int32_t* vo = T.vb[pass & 1];
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    int64_t i = base + r * 32 + lane;
    if (i < T.m) {
      uint32_t d = (key[r] >> shift) & (kRadixBins - 1);
      uint32_t pos = sbase[d] + cnt[warp][d] + rank[r];
      ko[pos] = key[r];
      vo[pos] = val[r];
    }
  }
}

__device__ __forceinline__ const uint32_t* sorted_keys(const TableWork& T, const DevHeader* h, int t) {
  return T.kb[(num_passes(h, t) - 1) & 1];
}

// Number of run starts (first row or key change) per tile of sorted keys.
__global__ void __launch_bounds__(kSortThreads) rle_count_kernel(TwoTables a) {
  int tile;
  int t = table_of_block(a, tile);
  const TableWork& T = a.t[t];
  const uint32_t* u = sorted_keys(T, a.h, t);
  int64_t base = static_cast<int64_t>(tile) * kSortTile;
  uint32_t c = 0;
  for (int it = 0; it < kSortItems; ++it) {
    int64_t i = base + it * kSortThreads + threadIdx.x;
    if (i < T.m && (i == 0 || u[i] != u[i - 1])) ++c;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  __shared__ uint32_t ws[kSortThreads / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t s = 0;
    for (int w = 0; w < kSortThreads / 32; ++w) s += ws[w];
    T.rle_cnt[tile] = s;
  }
}

// Writes perm, sorted keys, the run index of every sorted row, and the
// runs (key, offset).  Each thread owns kSortItems consecutive rows.
__global__ void __launch_bounds__(kSortThreads) rle_write_kernel(TwoTables a) {
  int tile;
  int t = table_of_block(a, tile);
  const TableWork& T = a.t[t];
  const DevHeader* h = a.h;
  int P = num_passes(h, t);
  const uint32_t* u = T.kb[(P - 1) & 1];
  const int32_t* v = T.vb[(P - 1) & 1];
  uint32_t kmin = h->kmin[t];
  __shared__ uint32_t s_red[kSortThreads / 32];
  __shared__ uint32_t s_prefix;
  // runs that start in earlier tiles
  uint32_t part = 0;
  for (int i = threadIdx.x; i < tile; i += blockDim.x) part += T.rle_cnt[i];
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t s = 0;
    for (int w = 0; w < kSortThreads / 32; ++w) s += s_red[w];
    s_prefix = s;
  }
  __syncthreads();
  int64_t base = static_cast<int64_t>(tile) * kSortTile + static_cast<int64_t>(threadIdx.x) * kSortItems;
  uint32_t flags = 0, c = 0;
  for (int it = 0; it < kSortItems; ++it) {
    int64_t i = base + it;
    if (i < T.m && (i == 0 || u[i] != u[i - 1])) {
      flags |= 1u << it;
      ++c;
    }
  }
  // block exclusive scan of c
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = c;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  __shared__ uint32_t s_w[kSortThreads / 32];
  __syncthreads();
  if (lane == 31) s_w[warp] = incl;
  __syncthreads();
  uint32_t wpre = 0;
  for (int w = 0; w < warp; ++w) wpre += s_w[w];
  int64_t run = static_cast<int64_t>(s_prefix) + wpre + incl - c - 1;  // run of the row before my first
  for (int it = 0; it < kSortItems; ++it) {
    int64_t i = base + it;
    if (i >= T.m) break;
    int32_t key = ordered_to_key(u[i] + kmin);
    if (flags & (1u << it)) {
      ++run;
      T.run_key[run] = key;
      T.run_off[run] = static_cast<int32_t>(i);
    }
    T.perm[i] = v[i];
    T.sorted_key[i] = key;
    T.seg[i] = static_cast<int32_t>(run);
    if (i == T.m - 1) {
      a.h->num_runs[t] = run + 1;
      T.run_off[run + 1] = static_cast<int32_t>(T.m);
    }
  }
}

__device__ __forceinline__ int64_t lower_bound_key(const int32_t* keys, int64_t n, int32_t k) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (keys[mid] < k)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// For every run of either table: the size of the run with the same key in
// the other table (0 if none) and the head slot of the key group (the run
// index on A's side).
__global__ void match_kernel(TwoTables a) {
  int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  DevHeader* h = a.h;
  const TableWork& A = a.t[0];
  const TableWork& B = a.t[1];
  int64_t UA = h->num_runs[0], UB = h->num_runs[1];
  if (i < UA) {
    int32_t k = A.run_key[i];
    int64_t j = lower_bound_key(B.run_key, UB, k);
    int32_t mine = A.run_off[i + 1] - A.run_off[i];
    A.hdslot[i] = static_cast<int32_t>(i);
    if (j < UB && B.run_key[j] == k) {
      int32_t other = B.run_off[j + 1] - B.run_off[j];
      A.other[i] = other;
      atomicAdd(reinterpret_cast<unsigned long long*>(&h->num_groups), 1ull);
      atomicAdd(reinterpret_cast<unsigned long long*>(&h->reduced_rows),
                static_cast<unsigned long long>(mine + other - 1));
    } else {
      A.other[i] = 0;
    }
  }
  if (i < UB) {
    int32_t k = B.run_key[i];
    int64_t j = lower_bound_key(A.run_key, UA, k);
    if (j < UA && A.run_key[j] == k) {
      B.other[i] = A.run_off[j + 1] - A.run_off[j];
      B.hdslot[i] = static_cast<int32_t>(j);
    } else {
      B.other[i] = 0;
      B.hdslot[i] = -1;
    }
  }
}

}  // namespace

cudaError_t launch_reset(const Plan& p, cudaStream_t s) {
  int n0 = p.t[0].chunks, n1 = p.t[1].chunks;
  int work = n0 > n1 ? n0 : n1;
  int blocks = (work + 255) / 256;
  if (blocks < 1) blocks = 1;
  if (blocks > 64) blocks = 64;
  uint32_t* s0 = p.t[0].chunk_status;
  uint32_t* s1 = p.t[1].chunk_status;
  reset_kernel<<<blocks, 256, 0, s>>>(p.hdr, s0, s0 ? n0 : 0, s1, s1 ? n1 : 0);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_grouping(const Plan& p, cudaStream_t s) {
  TwoTables a;
  a.t[0] = p.t[0];
  a.t[1] = p.t[1];
  a.h = p.hdr;
  a.nb0 = p.t[0].tiles;
  int nb = p.t[0].tiles + p.t[1].tiles;
  if (nb == 0) return cudaSuccess;
  key_range_kernel<<<nb, kSortThreads, 0, s>>>(a);
  for (int pass = 0; pass < kMaxPasses; ++pass) {
    radix_hist_kernel<<<nb, kSortThreads, 0, s>>>(a, pass);
    radix_scan_kernel<<<2, kScanThreads, 0, s>>>(a, pass);
    radix_scatter_kernel<<<nb, kSortThreads, 0, s>>>(a, pass);
  }
  rle_count_kernel<<<nb, kSortThreads, 0, s>>>(a);
  rle_write_kernel<<<nb, kSortThreads, 0, s>>>(a);
  int64_t mm = p.t[0].m > p.t[1].m ? p.t[0].m : p.t[1].m;
  int mb = static_cast<int>((mm + 255) / 256);
  if (mb > 0) match_kernel<<<mb, 256, 0, s>>>(a);
  count_launches(1 + 3 * kMaxPasses + 2 + (mb > 0 ? 1 : 0));
  return cudaGetLastError();
}

}  // namespace figaro
