// Key grouping of both tables: a stable LSD radix sort of (key, row index),
// run-length encoding of the sorted keys, and the matching of runs between
// the tables (the inner natural join keeps only keys present in both).
//
// The paper assumes inputs already sorted by the join attribute (Section 2,
// experimental setup); this step produces that order.  Stability keeps rows
// with equal keys in input order, which fixes the order of the QR tail rows
// inside each key group.
//
// Launches (each covers both tables; blocks [0, tiles_A) work on A; a tile
// is 8,192 keys):
//   1. key_hist:   the key range and each tile's counts of the first 8-bit
//                  digit of the order-preserving uint32 key.  Digits above the
//                  highest bit in which min and max differ are equal for every
//                  key, so only ceil(bits / 8) passes run; the kernels of the
//                  other passes return at once.
//   2. per pass, reduce-then-scan (no waiting between tiles):
//        tile_count  the tile's digit counts (passes after the first),
//        tile_scan   per digit, the exclusive scan over tiles plus the keys of
//                    smaller digits: each tile's output offset per digit,
//        sort_pass   stable ranking in shared memory (warp multi-split by
//                    ballots), keys staged in digit order, coalesced scatter.
//      The last pass writes the final perm / sorted keys.
//   3. run_count, runs: run starts per tile, then each tile's run index from
//                  the sum of the earlier tiles' counts; run keys, offsets,
//                  the run index of every sorted row, and a key lookup table.
//   4. match:      per run, the size of the run with the same key in the other
//                  table (lookup table, binary search outside its range) and
//                  the head slot of the key group.
#include "common.cuh"
#include "internal.h"

namespace figaro {
namespace {

struct TwoTables {
  TableWork t[2];
  DevHeader* h;
  int nb0;  // tiles of table 0
  int nb;   // tiles of both tables
  int64_t spin_limit;
  int64_t lut_size;  // entries of each table's key lookup table
};

__device__ __forceinline__ int table_of(const TwoTables& a, int g, int& tile) {
  if (g < a.nb0) {
    tile = g;
    return 0;
  }
  tile = g - a.nb0;
  return 1;
}

__device__ __forceinline__ int num_passes(const DevHeader* h, int t) {
  uint32_t d = h->kmin[t] ^ h->kmax[t];
  int bits = d ? 32 - __clz(d) : 0;
  int p = (bits + kRadixBits - 1) / kRadixBits;
  return p < 1 ? 1 : p;
}

// Per-tile digit counts and output offsets of a pass (reduce-then-scan),
// kept in the table's sort word area: [pass][counts | offsets][tile][digit].
__device__ __forceinline__ uint32_t* tile_counts(const TableWork& T, int pass) {
  return reinterpret_cast<uint32_t*>(T.sort_status) + static_cast<int64_t>(pass) * 2 * T.tiles * kRadixBins;
}
__device__ __forceinline__ uint32_t* tile_offsets(const TableWork& T, int pass) {
  return tile_counts(T, pass) + static_cast<int64_t>(T.tiles) * kRadixBins;
}

__global__ void reset_kernel(DevHeader* h, int report_rank) {
  pdl_enter();
  h->status = 0;
  h->report_rank = report_rank;
  h->dep_cols = 0;
  for (int i = 0; i < 8; ++i) h->ticket[i] = 0;
  h->kmin[0] = h->kmin[1] = 0xffffffffu;
  h->kmax[0] = h->kmax[1] = 0u;
  h->num_runs[0] = h->num_runs[1] = 0;
  h->num_groups = 0;
  h->reduced_rows = 0;
  h->jacobi_sweeps = 0;
  h->bar_count = 0u;
  h->bar_gen = 0u;
  h->sweep_any[0] = h->sweep_any[1] = h->sweep_any[2] = 0u;
}

// The key range, the first pass's digit counts per tile and their global
// sum (the later passes' counts come from tile_count_kernel, once the key
// range has fixed how many passes run).
__device__ __forceinline__ void key_hist_body(const TableWork& T, int t, DevHeader* h, int tile) {
  __shared__ uint32_t hist[kRadixBins];
  for (int i = threadIdx.x; i < kRadixBins; i += blockDim.x) hist[i] = 0u;
  __syncthreads();
  uint32_t lo = 0xffffffffu, hi = 0u;
  const int64_t base = static_cast<int64_t>(tile) * kSortTile;
  uint32_t u[kSortItems];
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {
    const int64_t i = base + it * kSortThreads + threadIdx.x;
    u[it] = i < T.m ? key_to_ordered(T.key[i]) : 0u;
  }
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {
    const int64_t i = base + it * kSortThreads + threadIdx.x;
    const bool valid = i < T.m;
    if (valid) {
      lo = min(lo, u[it]);
      hi = max(hi, u[it]);
    }
    if (valid) atomicAdd(&hist[u[it] & (kRadixBins - 1)], 1u);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&h->kmin[t], lo);
    atomicMax(&h->kmax[t], hi);
  }
  __syncthreads();
  uint32_t* tc = tile_counts(T, 0) + static_cast<int64_t>(tile) * kRadixBins;
  for (int d = threadIdx.x; d < kRadixBins; d += blockDim.x) {
    const uint32_t c = hist[d];
    tc[d] = c;
    if (c) atomicAdd(&T.hist[d], c);
  }
}

// Tables already in key order (FIGARO_FLAG_PRESORTED; the paper's setting,
// Section 2): the identity permutation, the keys as the sorted keys, the key
// range, and a check that the order holds (a table that is not in order
// sets kStatusUnsorted; the later steps stay in bounds either way).
__global__ void __launch_bounds__(kSortThreads) presorted_kernel(TwoTables a) {
  pdl_enter();
  int tile;
  const int t = table_of(a, blockIdx.x, tile);
  const TableWork& T = a.t[t];
  uint32_t lo = 0xffffffffu, hi = 0u;
  int bad = 0;
  const int64_t base = static_cast<int64_t>(tile) * kSortTile;
  for (int it = 0; it < kSortItems; ++it) {
    const int64_t i = base + it * kSortThreads + threadIdx.x;
    if (i < T.m) {
      const int32_t k = T.key[i];
      const uint32_t u = key_to_ordered(k);
      lo = min(lo, u);
      hi = max(hi, u);
      if (i > 0 && T.key[i - 1] > k) bad = 1;
      T.perm[i] = static_cast<int32_t>(i);
      T.sorted_key[i] = k;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (lo <= hi) {
      atomicMin(&a.h->kmin[t], lo);
      atomicMax(&a.h->kmax[t], hi);
    }
    if (bad) set_status(&a.h->status, kStatusUnsorted);
  }
}

__global__ void __launch_bounds__(kSortThreads) key_hist_kernel(TwoTables a) {
  pdl_enter();
  int tile;
  const int t = table_of(a, blockIdx.x, tile);
  key_hist_body(a.t[t], t, a.h, tile);
}

__global__ void __launch_bounds__(kSortThreads) key_hist_batched(BatchDev b, BatchJobs J) {
  pdl_enter();
  const int j = batch_job(J, blockIdx.x);
  const Plan& P = b.plans[J.inst[j]];
  key_hist_body(P.t[J.aux[j]], J.aux[j], P.hdr, blockIdx.x - J.first[j]);
}

// Digit counts of every tile for a later pass (the keys as the previous pass left them).
__device__ __forceinline__ void tile_count_body(const TableWork& T, int t, const DevHeader* h, int tile, int pass) {
  if (pass >= num_passes(h, t)) return;
  __shared__ uint32_t hist[kRadixBins];
  for (int d = threadIdx.x; d < kRadixBins; d += blockDim.x) hist[d] = 0u;
  __syncthreads();
  const uint32_t* kin = T.kb[(pass - 1) & 1];
  const int shift = pass * kRadixBits;
  const int64_t base = static_cast<int64_t>(tile) * kSortTile;
  uint32_t u[kSortItems];
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {
    const int64_t i = base + it * kSortThreads + threadIdx.x;
    u[it] = i < T.m ? kin[i] : 0u;
  }
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {
    const int64_t i = base + it * kSortThreads + threadIdx.x;
    const bool valid = i < T.m;
    if (valid) atomicAdd(&hist[(u[it] >> shift) & (kRadixBins - 1)], 1u);
  }
  __syncthreads();
  uint32_t* tc = tile_counts(T, pass) + static_cast<int64_t>(tile) * kRadixBins;
  for (int d = threadIdx.x; d < kRadixBins; d += blockDim.x) {
    const uint32_t c = hist[d];
    tc[d] = c;
    if (c) atomicAdd(&T.hist[pass * kRadixBins + d], c);  // the pass's global counts
  }
}

__global__ void __launch_bounds__(kSortThreads) tile_count_kernel(TwoTables a, int pass) {
  pdl_enter();
  int tile;
  const int t = table_of(a, blockIdx.x, tile);
  tile_count_body(a.t[t], t, a.h, tile, pass);
}

__global__ void __launch_bounds__(kSortThreads) tile_count_batched(BatchDev b, BatchJobs J, int pass) {
  pdl_enter();
  const int j = batch_job(J, blockIdx.x);
  const Plan& P = b.plans[J.inst[j]];
  tile_count_body(P.t[J.aux[j]], J.aux[j], P.hdr, blockIdx.x - J.first[j], pass);
}

// Per (table, digit): the position of each tile's first key of that digit in
// the pass's output, = (keys of smaller digits) + (keys of this digit in
// earlier tiles): an exclusive scan over tiles.
__device__ __forceinline__ void tile_scan_body(const TableWork& T, int t, const DevHeader* h, int d, int pass) {
  if (T.tiles == 0 || pass >= num_passes(h, t)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ uint32_t s_w[kRadixBins / 32];
  __shared__ uint32_t s_carry;
  // keys of digits below d
  uint32_t v = threadIdx.x < d ? T.hist[pass * kRadixBins + threadIdx.x] : 0u;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) s_w[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t g = 0;
    for (int w = 0; w < kRadixBins / 32; ++w) g += s_w[w];
    s_carry = g;
  }
  __syncthreads();
  const uint32_t* tc = tile_counts(T, pass);
  uint32_t* to = tile_offsets(T, pass);
  for (int c0 = 0; c0 < T.tiles; c0 += kRadixBins) {
    const int tile = c0 + threadIdx.x;
    const uint32_t x = tile < T.tiles ? tc[static_cast<int64_t>(tile) * kRadixBins + d] : 0u;
    uint32_t incl = x;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    __syncthreads();
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    uint32_t before = s_carry;
    for (int w = 0; w < warp; ++w) before += s_w[w];
    if (tile < T.tiles) to[static_cast<int64_t>(tile) * kRadixBins + d] = before + incl - x;
    __syncthreads();
    if (threadIdx.x == kRadixBins - 1) s_carry = before + incl;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kRadixBins) tile_scan_kernel(TwoTables a, int pass) {
  pdl_enter();
  const int t = blockIdx.x / kRadixBins;
  tile_scan_body(a.t[t], t, a.h, blockIdx.x % kRadixBins, pass);
}

// Batched form: one CTA per table job (a batch's tables have few tiles),
// thread d walks digit d's tile counts in order from the keys of the smaller
// digits (a block-wide exclusive scan of the pass's histogram).
__global__ void __launch_bounds__(kRadixBins) tile_scan_batched(BatchDev b, BatchJobs J, int pass) {
  pdl_enter();
  const int j = blockIdx.x;
  const Plan& P = b.plans[J.inst[j]];
  const int t = J.aux[j];
  const TableWork& T = P.t[t];
  if (T.tiles == 0 || pass >= num_passes(P.hdr, t)) return;
  const int d = threadIdx.x, lane = d & 31, warp = d >> 5;
  __shared__ uint32_t s_w[kRadixBins / 32];
  const uint32_t h = T.hist[pass * kRadixBins + d];
  uint32_t incl = h;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_w[warp] = incl;
  __syncthreads();
  uint32_t run = incl - h;
  for (int w = 0; w < warp; ++w) run += s_w[w];
  const uint32_t* tc = tile_counts(T, pass);
  uint32_t* to = tile_offsets(T, pass);
  for (int tile = 0; tile < T.tiles; ++tile) {
    const uint32_t x = tc[static_cast<int64_t>(tile) * kRadixBins + d];
    to[static_cast<int64_t>(tile) * kRadixBins + d] = run;
    run += x;
  }
}

// One stable LSD pass over digit `pass` (the scatter of reduce-then-scan).
// Each tile ranks its keys stably (warp multi-split with match_any, then a
// prefix over warps), places keys and payloads in shared memory in digit
// order, and writes them out so that consecutive threads write consecutive
// positions of each digit's output run (coalesced), at the digit offsets
// from tile_scan_kernel.
constexpr int kSortSmem = (kSortThreads / 32) * kRadixBins * 4 + 3 * kRadixBins * 4 + 2 * kSortTile * 4;

__device__ __forceinline__ void sort_pass_body(const TableWork& T, int t, const DevHeader* h, int tile, int pass) {
  constexpr int kWarps = kSortThreads / 32;
  extern __shared__ __align__(16) uint32_t sm_sort[];
  uint32_t (*cnt)[kRadixBins] = reinterpret_cast<uint32_t (*)[kRadixBins]>(sm_sort);
  uint32_t* sbase = sm_sort + kWarps * kRadixBins;   // output offset of the tile's first key of digit d
  uint32_t* tpre = sbase + kRadixBins;               // tile-local start of digit d
  uint32_t* s_w = tpre + kRadixBins;                 // per-warp sums of the local scan
  uint32_t* sk = s_w + kRadixBins;                   // keys in digit order
  int32_t* sv = reinterpret_cast<int32_t*>(sk + kSortTile);  // payloads in digit order
  const int P = num_passes(h, t);
  if (pass >= P) return;
  const bool last = pass == P - 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kWarps * kRadixBins; i += blockDim.x) (&cnt[0][0])[i] = 0u;
  __syncthreads();
  const int shift = pass * kRadixBits;
  const int64_t tile0 = static_cast<int64_t>(tile) * kSortTile;
  const int64_t base = tile0 + warp * (32 * kSortItems);
  const uint32_t* kin = pass == 0 ? nullptr : T.kb[(pass - 1) & 1];
  const int32_t* vin = pass == 0 ? nullptr : T.vb[(pass - 1) & 1];
  uint32_t key[kSortItems];
  uint32_t rank[kSortItems];
  const uint32_t lt_mask = (1u << lane) - 1u;
  // all loads first (the warp barriers of the ranking would serialise them)
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const int64_t i = base + r * 32 + lane;
    key[r] = i < T.m ? (pass == 0 ? key_to_ordered(T.key[i]) : kin[i]) : 0u;
  }
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const int64_t i = base + r * 32 + lane;
    const bool valid = i < T.m;
    const uint32_t u = key[r];
    const uint32_t d = valid ? ((u >> shift) & (kRadixBins - 1)) : kRadixBins;  // padding gets its own bin
    // lanes with the same digit: the AND over the digit's 9 bits of the
    // matching ballot (the padding bin 256 needs the ninth bit)
    uint32_t peers = 0xffffffffu;
#pragma unroll
    for (int bit = 0; bit <= kRadixBits; ++bit) {
      const uint32_t m = __ballot_sync(0xffffffffu, (d >> bit) & 1u);
      peers &= ((d >> bit) & 1u) ? m : ~m;
    }
    uint32_t before = 0;
    if (valid) before = cnt[warp][d];
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) cnt[warp][d] = before + __popc(peers);
    __syncwarp();
    rank[r] = before + __popc(peers & lt_mask);
  }
  __syncthreads();
  // per digit: exclusive prefix over warps, the digit's total in the tile,
  // its tile-local start (scan over digits) and the output offset
  uint32_t tot = 0;
  if (threadIdx.x < kRadixBins) {
    const int d = threadIdx.x;
    for (int w = 0; w < kWarps; ++w) {
      const uint32_t c = cnt[w][d];
      cnt[w][d] = tot;
      tot += c;
    }
    uint32_t incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_w[warp] = incl;
    tpre[d] = incl - tot;  // within-warp part; the earlier warps are added below
    sbase[d] = tile_offsets(T, pass)[static_cast<int64_t>(tile) * kRadixBins + d];
  }
  __syncthreads();
  if (threadIdx.x < kRadixBins) {
    uint32_t add = 0;
    for (int w = 0; w < warp; ++w) add += s_w[w];
    tpre[threadIdx.x] += add;
  }
  __syncthreads();
  // keys and payloads into shared memory in digit order
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const int64_t i = base + r * 32 + lane;
    if (i < T.m) {
      const uint32_t d = (key[r] >> shift) & (kRadixBins - 1);
      const uint32_t lpos = tpre[d] + cnt[warp][d] + rank[r];
      sk[lpos] = key[r];
      sv[lpos] = pass == 0 ? static_cast<int32_t>(i) : vin[i];  // the payload is read again (cached)
    }
  }
  __syncthreads();
  // coalesced writes: position j of the tile's digit-ordered keys goes to
  // sbase[d] + (j - tpre[d])
  const int cnt_tile = static_cast<int>(T.m - tile0 < kSortTile ? T.m - tile0 : kSortTile);
  uint32_t* ko = T.kb[pass & 1];
  int32_t* vo = last ? T.perm : T.vb[pass & 1];
  for (int j = threadIdx.x; j < cnt_tile; j += kSortThreads) {
    const uint32_t k = sk[j];
    const uint32_t d = (k >> shift) & (kRadixBins - 1);
    const uint32_t pos = sbase[d] + (static_cast<uint32_t>(j) - tpre[d]);
    if (last) {
      T.sorted_key[pos] = ordered_to_key(k);
    } else {
      ko[pos] = k;
    }
    vo[pos] = sv[j];
  }
}

__global__ void __launch_bounds__(kSortThreads, 2) sort_pass_kernel(TwoTables a, int pass) {
  pdl_enter();
  int tile;
  const int t = table_of(a, blockIdx.x, tile);
  sort_pass_body(a.t[t], t, a.h, tile, pass);
}

__global__ void __launch_bounds__(kSortThreads, 2) sort_pass_batched(BatchDev b, BatchJobs J, int pass) {
  pdl_enter();
  const int j = batch_job(J, blockIdx.x);
  const Plan& P = b.plans[J.inst[j]];
  sort_pass_body(P.t[J.aux[j]], J.aux[j], P.hdr, blockIdx.x - J.first[j], pass);
}

// Run starts per tile of the sorted keys (a row starts a run when its key
// differs from the row before it).
__device__ __forceinline__ void run_count_body(const TableWork& T, int tile) {
  const int64_t base = static_cast<int64_t>(tile) * kSortTile;
  uint32_t c = 0;
  for (int it = 0; it < kSortItems; ++it) {
    const int64_t i = base + it * kSortThreads + threadIdx.x;
    if (i < T.m && (i == 0 || T.sorted_key[i] != T.sorted_key[i - 1])) ++c;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  __shared__ uint32_t s_w[kSortThreads / 32];
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t tot = 0;
    for (int w = 0; w < kSortThreads / 32; ++w) tot += s_w[w];
    reinterpret_cast<uint32_t*>(T.run_status)[tile] = tot;
  }
}

__global__ void __launch_bounds__(kSortThreads) run_count_kernel(TwoTables a) {
  pdl_enter();
  int tile;
  const int t = table_of(a, blockIdx.x, tile);
  run_count_body(a.t[t], tile);
}

__global__ void __launch_bounds__(kSortThreads) run_count_batched(BatchDev b, BatchJobs J) {
  pdl_enter();
  const int j = batch_job(J, blockIdx.x);
  run_count_body(b.plans[J.inst[j]].t[J.aux[j]], blockIdx.x - J.first[j]);
}

// Runs of the sorted keys: run keys, run offsets, the run index of every
// sorted row, and each run start's slot in the key lookup table.  The number
// of runs before the tile is the sum of the earlier tiles' counts (a block
// reduction, no waiting).  Rows are staged through shared memory so that
// global accesses stay coalesced.
__device__ __forceinline__ void runs_body(const TableWork& T, int t, DevHeader* h, int tile, int64_t lut_size) {
  __shared__ int32_t sk[kSortTile + 1];
  __shared__ uint32_t s_w[kSortThreads / 32];
  __shared__ uint64_t s_excl;
  const int64_t base = static_cast<int64_t>(tile) * kSortTile;
  const int64_t m = T.m;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // runs in the earlier tiles
  {
    const uint32_t* counts = reinterpret_cast<const uint32_t*>(T.run_status);
    uint64_t e = 0;
    for (int j = threadIdx.x; j < tile; j += kSortThreads) e += counts[j];
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    __shared__ uint64_t s_e[kSortThreads / 32];
    if (lane == 0) s_e[warp] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint64_t tot = 0;
      for (int w = 0; w < kSortThreads / 32; ++w) tot += s_e[w];
      s_excl = tot;
    }
  }
  for (int e = threadIdx.x; e < kSortTile + 1; e += blockDim.x) {
    const int64_t i = base - 1 + e;
    sk[e] = (i >= 0 && i < m) ? T.sorted_key[i] : 0;
  }
  __syncthreads();
  // flags of my kSortItems consecutive rows
  const int r0 = threadIdx.x * kSortItems;
  uint32_t flags = 0, c = 0;
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {
    const int64_t i = base + r0 + it;
    if (i < m && (i == 0 || sk[r0 + it + 1] != sk[r0 + it])) {
      flags |= 1u << it;
      ++c;
    }
  }
  uint32_t incl = c;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_w[warp] = incl;
  __syncthreads();
  uint32_t wpre = 0;
  for (int w = 0; w < warp; ++w) wpre += s_w[w];
  const uint32_t kbase = min(h->kmin[0], h->kmin[1]);
  int64_t run = static_cast<int64_t>(s_excl) + wpre + incl - c - 1;  // run of the row before my first
  int32_t segs[kSortItems];
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {
    const int64_t i = base + r0 + it;
    if (flags & (1u << it)) {
      ++run;
      const int32_t k = sk[r0 + it + 1];
      T.run_key[run] = k;
      T.run_off[run] = static_cast<int32_t>(i);
      const uint32_t off = key_to_ordered(k) - kbase;
      if (off < static_cast<uint32_t>(lut_size)) T.lut[off] = static_cast<int32_t>(run);
    }
    segs[it] = static_cast<int32_t>(run);
    if (i == m - 1) {
      h->num_runs[t] = run + 1;
      T.run_off[run + 1] = static_cast<int32_t>(m);
    }
  }
  __syncthreads();  // reuse sk for the run indices, written back coalesced
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) sk[r0 + it] = segs[it];
  __syncthreads();
  for (int e = threadIdx.x; e < kSortTile; e += blockDim.x) {
    const int64_t i = base + e;
    if (i < m) T.seg[i] = sk[e];
  }
}

__global__ void __launch_bounds__(kSortThreads) runs_kernel(TwoTables a) {
  pdl_enter();
  int tile;
  const int t = table_of(a, blockIdx.x, tile);
  runs_body(a.t[t], t, a.h, tile, a.lut_size);
}

__global__ void __launch_bounds__(kSortThreads) runs_batched(BatchDev b, BatchJobs J) {
  pdl_enter();
  const int j = batch_job(J, blockIdx.x);
  const Plan& P = b.plans[J.inst[j]];
  runs_body(P.t[J.aux[j]], J.aux[j], P.hdr, blockIdx.x - J.first[j], P.lut_size);
}

__device__ __forceinline__ int64_t lower_bound_key(const int32_t* keys, int64_t n, int32_t k) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (keys[mid] < k)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// For every run of either table: the size of the run with the same key in
// the other table (0 if none) and the head slot of the key group (the run
// index on A's side), also packed with the run's row range into one 16-byte
// record for the head/tail step.
// The run of key k in table O: the lookup table when k is inside its range
// (an entry is trusted only if it names a run with that key: no entry needs
// initialising), else a binary search of O's run keys.
__device__ __forceinline__ int64_t find_run(const DevHeader* h, int64_t lut_size, const TableWork& O, int64_t UO,
                                            int32_t k) {
  const uint32_t off = key_to_ordered(k) - min(h->kmin[0], h->kmin[1]);
  if (off < static_cast<uint32_t>(lut_size)) {
    const int64_t j = O.lut[off];
    return (j >= 0 && j < UO && O.run_key[j] == k) ? j : -1;
  }
  const int64_t j = lower_bound_key(O.run_key, UO, k);
  return (j < UO && O.run_key[j] == k) ? j : -1;
}

__device__ __forceinline__ void match_body(const TableWork& A, const TableWork& B, DevHeader* h, int64_t lut_size,
                                           int block) {
  const int64_t i = static_cast<int64_t>(block) * blockDim.x + threadIdx.x;
  const int64_t UA = h->num_runs[0], UB = h->num_runs[1];
  unsigned long long groups = 0, reduced = 0;
  if (i < UA) {
    const int32_t k = A.run_key[i];
    const int64_t j = find_run(h, lut_size, B, UB, k);
    const int32_t mine = A.run_off[i + 1] - A.run_off[i];
    A.hdslot[i] = static_cast<int32_t>(i);
    int32_t other = 0;
    if (j >= 0) {
      other = B.run_off[j + 1] - B.run_off[j];
      groups = 1;
      reduced = static_cast<unsigned long long>(mine + other - 1);
    }
    A.other[i] = other;
    reinterpret_cast<int4*>(A.run_info)[i] = make_int4(A.run_off[i], A.run_off[i + 1], other, static_cast<int32_t>(i));
  }
  // one atomic per warp for the counts of key groups and reduced rows
  for (int o = 16; o > 0; o >>= 1) {
    groups += __shfl_xor_sync(0xffffffffu, groups, o);
    reduced += __shfl_xor_sync(0xffffffffu, reduced, o);
  }
  if ((threadIdx.x & 31) == 0 && groups) {
    atomicAdd(reinterpret_cast<unsigned long long*>(&h->num_groups), groups);
    atomicAdd(reinterpret_cast<unsigned long long*>(&h->reduced_rows), reduced);
  }
  if (i < UB) {
    const int32_t k = B.run_key[i];
    const int64_t j = find_run(h, lut_size, A, UA, k);
    int32_t other = 0, slot = -1;
    if (j >= 0) {
      other = A.run_off[j + 1] - A.run_off[j];
      slot = static_cast<int32_t>(j);
    }
    B.other[i] = other;
    B.hdslot[i] = slot;
    reinterpret_cast<int4*>(B.run_info)[i] = make_int4(B.run_off[i], B.run_off[i + 1], other, slot);
  }
}

__global__ void match_kernel(TwoTables a) {
  pdl_enter(); match_body(a.t[0], a.t[1], a.h, a.lut_size, blockIdx.x); }

__global__ void match_batched(BatchDev b, BatchJobs J) {
  pdl_enter();
  const int j = batch_job(J, blockIdx.x);
  const Plan& P = b.plans[J.inst[j]];
  match_body(P.t[0], P.t[1], P.hdr, P.lut_size, blockIdx.x - J.first[j]);
}

// Reset of every instance's header and digit histograms (one CTA each).
__global__ void batch_reset_kernel(BatchDev b) {
  pdl_enter();
  const Plan& P = b.plans[blockIdx.x];
  if (threadIdx.x == 0) {
    DevHeader* h = P.hdr;
    h->status = 0;
    h->report_rank = P.report_rank;
    h->dep_cols = 0;
    for (int i = 0; i < 8; ++i) h->ticket[i] = 0;
    h->kmin[0] = h->kmin[1] = 0xffffffffu;
    h->kmax[0] = h->kmax[1] = 0u;
    h->num_runs[0] = h->num_runs[1] = 0;
    h->num_groups = 0;
    h->reduced_rows = 0;
    h->jacobi_sweeps = 0;
    h->bar_count = 0u;
    h->bar_gen = 0u;
    h->sweep_any[0] = h->sweep_any[1] = h->sweep_any[2] = 0u;
  }
  for (int t = 0; t < 2; ++t)
    if (P.t[t].m > 0)
      for (int i = threadIdx.x; i < kMaxPasses * kRadixBins; i += blockDim.x) P.t[t].hist[i] = 0u;
}

}  // namespace

cudaError_t launch_batch_grouping(const BatchDev& b, const BatchJobs& tiles, const BatchJobs& match, cudaStream_t s) {
  pdl_launch(batch_reset_kernel, b.count, 256, 0, s, b);
  count_launches(1);
  if (tiles.njobs > 0) {
    static int granted[64] = {0};
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (dev < 0 || dev >= 64 || !granted[dev]) {
      err = cudaFuncSetAttribute(sort_pass_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, kSortSmem);
      if (err != cudaSuccess) return err;
      if (dev >= 0 && dev < 64) granted[dev] = 1;
    }
    pdl_launch(key_hist_batched, tiles.ctas, kSortThreads, 0, s, b, tiles);
    for (int pass = 0; pass < kMaxPasses; ++pass) {
      if (pass > 0) pdl_launch(tile_count_batched, tiles.ctas, kSortThreads, 0, s, b, tiles, pass);
      pdl_launch(tile_scan_batched, tiles.njobs, kRadixBins, 0, s, b, tiles, pass);
      pdl_launch(sort_pass_batched, tiles.ctas, kSortThreads, kSortSmem, s, b, tiles, pass);
    }
    pdl_launch(run_count_batched, tiles.ctas, kSortThreads, 0, s, b, tiles);
    pdl_launch(runs_batched, tiles.ctas, kSortThreads, 0, s, b, tiles);
    count_launches(3 + 3 * kMaxPasses - 1);
  }
  if (match.njobs > 0) {
    pdl_launch(match_batched, match.ctas, 256, 0, s, b, match);
    count_launches(1);
  }
  return cudaGetLastError();
}

// Words of the grouping step per table: per-tile digit counts and offsets of
// every pass (kMaxPasses x tiles x bins 64-bit words), and per-tile run counts.
int64_t group_status_words(int tiles) {
  return static_cast<int64_t>(kMaxPasses) * tiles * kRadixBins + tiles;
}

cudaError_t launch_reset(const Plan& p, cudaStream_t s) {
  // the header; the sort's per-tile counts and offsets and the run counts are
  // rewritten by every call
  pdl_launch(reset_kernel, 1, 1, 0, s, p.hdr, p.report_rank);
  count_launches(1);
  // the histograms are accumulated with atomics: clear them too
  for (int t = 0; t < 2; ++t)
    if (p.t[t].m > 0) {
      cudaError_t e = cudaMemsetAsync(p.t[t].hist, 0, sizeof(uint32_t) * kMaxPasses * kRadixBins, s);
      if (e != cudaSuccess) return e;
    }
  return cudaGetLastError();
}

cudaError_t launch_grouping(const Plan& p, cudaStream_t s) {
  TwoTables a;
  a.t[0] = p.t[0];
  a.t[1] = p.t[1];
  a.h = p.hdr;
  a.nb0 = p.t[0].tiles;
  a.nb = p.t[0].tiles + p.t[1].tiles;
  a.spin_limit = p.spin_limit;
  a.lut_size = p.lut_size;
  if (a.nb == 0) return cudaSuccess;
  static int granted[64] = {0};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 0 || dev >= 64 || !granted[dev]) {
    err = cudaFuncSetAttribute(sort_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSortSmem);
    if (err != cudaSuccess) return err;
    if (dev >= 0 && dev < 64) granted[dev] = 1;
  }
  if (p.presorted) {
    pdl_launch(presorted_kernel, a.nb, kSortThreads, 0, s, a);
    count_launches(1);
  } else {
    pdl_launch(key_hist_kernel, a.nb, kSortThreads, 0, s, a);
    // passes past the key range's highest differing digit return at once
    for (int pass = 0; pass < kMaxPasses; ++pass) {
      if (pass > 0) pdl_launch(tile_count_kernel, a.nb, kSortThreads, 0, s, a, pass);
      pdl_launch(tile_scan_kernel, 2 * kRadixBins, kRadixBins, 0, s, a, pass);
      pdl_launch(sort_pass_kernel, a.nb, kSortThreads, kSortSmem, s, a, pass);
    }
    count_launches(1 + 3 * kMaxPasses - 1);
  }
  pdl_launch(run_count_kernel, a.nb, kSortThreads, 0, s, a);
  pdl_launch(runs_kernel, a.nb, kSortThreads, 0, s, a);
  const int64_t mm = p.t[0].m > p.t[1].m ? p.t[0].m : p.t[1].m;
  const int mb = static_cast<int>((mm + 255) / 256);
  if (mb > 0) pdl_launch(match_kernel, mb, 256, 0, s, a);
  count_launches(2 + (mb > 0 ? 1 : 0));
  return cudaGetLastError();
}

}  // namespace figaro
