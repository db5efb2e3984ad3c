// Wide joins: n1 + n2 in (128, 512], each table at most 256 columns.  The
// CholeskyQR2 of the reduced matrix and the singular values of R, with the
// n x n work spread over many CTAs instead of one (the narrow path keeps an
// n x n matrix in one CTA's shared memory, which stops at n = 128).
//
// Gram products (the reduced matrix M = [head rows; A tails; B tails] of
// Claim 1, Section 1; CholeskyQR2 as on the narrow path):
//   * wide_form_kernel    pass 2: Q = X W for each block, written to memory
//                         (W = R1^{-1} is upper triangular, so the A tails
//                         use W[0:n1, :], the B tails W[n1:, n1:] and the
//                         head rows all of W);
//   * wide_gram_kernel    one job per (block, 64 x 64 upper tile of the
//                         block's Gram, row split): the tile's sum over the
//                         split's rows, register-tiled on CUDA cores, FP32
//                         partial sums flushed into FP64 every 256 rows on
//                         the mixed path, FP64 throughout on the plain path;
//   * wide_reduce_kernel  G = the sum of the partials in a fixed order
//                         (bitwise reproducible).
// Dense n x n steps, each one cooperative launch whose CTAs meet at grid
// barriers (the Jacobi: per-block waits between rounds) with bounded waits:
//   * wide_chol_first_kernel   blocked right-looking semi-definite Cholesky
//                              of G1 (32-column panels; a pivot below
//                              rank_tol * G1_kk marks the column dependent,
//                              its row of R1 is zero), then W = R1^{-1} one
//                              column per warp;
//   * wide_chol_second_kernel  mixed path: X = R1 + R1 (I - W R1), the FP64
//                              Newton step that makes X the inverse of the W
//                              the Grams used; R2 = chol(G2); R = R2 X in FP64
//                              (Section 1: R with R^T R = J^T J);
//   * wide_jacobi_kernel       one-sided Jacobi on the columns of R (Section
//                              3: sigma(J) = sigma(R)) by blocks of w columns:
//                              in each round the CTAs take disjoint pairs of
//                              blocks and run one cyclic sweep over the 2w
//                              columns of their pair, on the pair's Gram in
//                              shared memory, then apply the accumulated
//                              rotation to U and V;
//   * wide_sigma_kernel, wide_sort_kernel  sigma_j = ||R v_j|| / ||v_j|| in
//                              FP64 (mixed; ||u_j|| for sigma_j below 1e-3
//                              sigma_max) or ||u_j|| (plain), descending.
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace figaro {
namespace {

constexpr int kWT = 64;           // Gram / formation tile width
constexpr int kWRows = 32;        // rows per Gram chunk
constexpr int kWFlushChunks = 8;  // FP32 partial sums span at most 256 rows
constexpr int kWThreads = 256;
constexpr int kPanel = 32;        // Cholesky panel width

// ---------------------------------------------------------------- Gram ----

struct WideBlock {
  const void* X;            // rows x k (Gram input: rows x kout), leading dimension ldx
  int64_t ldx;
  int k;                    // input width (formation)
  int kout;                 // Gram width
  int off;                  // diagonal offset of the block's Gram inside G
  int w0;                   // formation uses W[w0:w0+k, w0:w0+kout]
  int64_t rows;             // host bound on the rows
  const int64_t* rows_dev;  // device row count (head rows), or null
  int tiles;                // ceil(kout / 64)
  int ntiles;               // upper tiles
  int splits;               // row splits of the Gram
  int64_t split_rows;
  int job0, njobs;          // Gram jobs
  void* Q;                  // formation output (rows x kout)
  int fjob0, fjobs;         // formation jobs: row tiles x column tiles
  // the engine that computes the block's Gram: CUDA cores (the fields above;
  // njobs = 0 when the tensor cores do it) or the tensor-core tile Gram
  int tc;                   // 1: tensor cores (FP32 input, mixed path)
  int tc_tiles, tc_splits, tc_njobs;
  int64_t tc_split_rows;
  // partials of the block as the reduce reads them: tw x tw doubles per job,
  // rtiles x (rtiles + 1) / 2 tiles of rsplits jobs from pbase (doubles)
  int tw, rtiles, rsplits;
  int64_t pbase;
};

struct WideArgs {
  WideBlock b[3];
  int gram_jobs, form_jobs;
  double* part;
  const void* W;
  int wld;
  double* G;
  int n;
};

__device__ __forceinline__ void upper_tile(int t, int T, int& ti, int& tj) {
  ti = 0;
  int len = T;
  while (t >= len) {
    t -= len;
    ++ti;
    --len;
  }
  tj = ti + t;
}

__device__ __forceinline__ int upper_index(int ti, int tj, int T) { return ti * T - ti * (ti - 1) / 2 + (tj - ti); }

__device__ __forceinline__ int64_t block_rows(const WideBlock& B) {
  if (!B.rows_dev) return B.rows;
  const int64_t r = *B.rows_dev;
  return r < B.rows ? r : B.rows;
}

template <typename T>
__global__ void __launch_bounds__(kWThreads) wide_gram_kernel(WideArgs a) {
  pdl_enter();
  // rows per chunk: 32 (FP32) or 16 (FP64), two buffers each for the two column blocks
  constexpr int RC = sizeof(T) == 4 ? kWRows : kWRows / 2;
  constexpr int PER = RC * kWT / kWThreads;  // elements of a chunk each thread stages
  __shared__ __align__(16) T xi[2][RC][kWT];
  __shared__ __align__(16) T xj[2][RC][kWT];
  int b = 0;
  while (b < 2 && static_cast<int>(blockIdx.x) >= a.b[b].job0 + a.b[b].njobs) ++b;
  const WideBlock& B = a.b[b];
  const int r = static_cast<int>(blockIdx.x) - B.job0;
  const int tile = r / B.splits, split = r - tile * B.splits;
  int ti, tj;
  upper_tile(tile, B.tiles, ti, tj);
  const int64_t rows = block_rows(B);
  const int64_t r0 = static_cast<int64_t>(split) * B.split_rows;
  const int64_t r1 = r0 + B.split_rows < rows ? r0 + B.split_rows : rows;
  const int ci0 = ti * kWT, cj0 = tj * kWT;
  const bool two = ti != tj;
  const T* X = static_cast<const T*>(B.X);
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  T acc[4][4];
  double tot[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      acc[i][j] = T(0);
      tot[i][j] = 0.0;
    }
  // the next chunk is read into registers while the current one is used
  T ri[PER], rj[PER];
  auto fetch = [&](int64_t c0) {
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int e = tid + q * kWThreads, rr = e / kWT, cc = e - rr * kWT;
      const int64_t row = c0 + rr;
      const bool in = row < r1;
      ri[q] = (in && ci0 + cc < B.kout) ? X[row * B.ldx + ci0 + cc] : T(0);
      rj[q] = (two && in && cj0 + cc < B.kout) ? X[row * B.ldx + cj0 + cc] : T(0);
    }
  };
  auto stage = [&](int buf) {
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int e = tid + q * kWThreads, rr = e / kWT, cc = e - rr * kWT;
      xi[buf][rr][cc] = ri[q];
      if (two) xj[buf][rr][cc] = rj[q];
    }
  };
  if (r0 < r1) {
    fetch(r0);
    stage(0);
  }
  __syncthreads();
  int chunk = 0, buf = 0;
  for (int64_t c0 = r0; c0 < r1; c0 += RC) {
    const bool more = c0 + RC < r1;
    if (more) fetch(c0 + RC);
    const T(*yi)[kWT] = xi[buf];
    const T(*yj)[kWT] = two ? xj[buf] : xi[buf];
#pragma unroll 4
    for (int rr = 0; rr < RC; ++rr) {
      T u[4], v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        u[q] = yi[rr][ty * 4 + q];
        v[q] = yj[rr][tx * 4 + q];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += u[i] * v[j];
    }
    // the other buffer was last read before the previous barrier
    if (more) stage(buf ^ 1);
    __syncthreads();
    buf ^= 1;
    if (sizeof(T) == 4 && ++chunk == kWFlushChunks) {
      chunk = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          tot[i][j] += static_cast<double>(acc[i][j]);
          acc[i][j] = T(0);
        }
    }
  }
  double* out = a.part + static_cast<int64_t>(blockIdx.x) * kWT * kWT;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) out[(ty * 4 + i) * kWT + tx * 4 + j] = tot[i][j] + static_cast<double>(acc[i][j]);
}

// G (n x n, both triangles) = sum over blocks and row splits of the tile
// partials, splits in ascending order.
__global__ void __launch_bounds__(kWThreads) wide_reduce_kernel(WideArgs a) {
  pdl_enter();
  const int64_t e = static_cast<int64_t>(blockIdx.x) * kWThreads + threadIdx.x;
  const int n = a.n;
  if (e >= static_cast<int64_t>(n) * n) return;
  const int i = static_cast<int>(e / n), j = static_cast<int>(e - static_cast<int64_t>(i) * n);
  const int lo = i < j ? i : j, hi = i < j ? j : i;
  double tot = 0.0;
  for (int b = 0; b < 3; ++b) {
    const WideBlock& B = a.b[b];
    if (B.rsplits == 0 || lo < B.off || hi >= B.off + B.kout) continue;
    const int ii = lo - B.off, jj = hi - B.off, tw = B.tw;
    const int ti = ii / tw, tj = jj / tw;
    const int64_t tt = static_cast<int64_t>(tw) * tw;
    const double* p = a.part + B.pbase + static_cast<int64_t>(upper_index(ti, tj, B.rtiles)) * B.rsplits * tt +
                      (ii % tw) * tw + (jj % tw);
    double t0 = 0.0, t1 = 0.0;
    int s = 0;
    for (; s + 1 < B.rsplits; s += 2) {
      t0 += p[static_cast<int64_t>(s) * tt];
      t1 += p[static_cast<int64_t>(s + 1) * tt];
    }
    if (s < B.rsplits) t0 += p[static_cast<int64_t>(s) * tt];
    tot += t0 + t1;
  }
  a.G[e] = tot;
}

// Q = X W[w0:w0+k, w0:w0+kout] for one 64 x 64 tile of Q (W upper triangular:
// column c of Q sums the input columns 0..c).
template <typename T>
__global__ void __launch_bounds__(kWThreads) wide_form_kernel(WideArgs a) {
  pdl_enter();
  __shared__ __align__(16) T xs[kWT][kPanel + 1];
  __shared__ __align__(16) T ws[kPanel][kWT];
  int b = 0;
  while (b < 2 && static_cast<int>(blockIdx.x) >= a.b[b].fjob0 + a.b[b].fjobs) ++b;
  const WideBlock& B = a.b[b];
  const int r = static_cast<int>(blockIdx.x) - B.fjob0;
  const int ct = r % B.tiles;
  const int64_t rt = r / B.tiles;
  const int64_t rows = block_rows(B);
  const int64_t row0 = rt * kWT;
  if (row0 >= rows) return;
  const int c0 = ct * kWT;
  const T* X = static_cast<const T*>(B.X);
  const T* W = static_cast<const T*>(a.W);
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  const int lend = (c0 + kWT < B.k ? c0 + kWT : B.k);  // input columns past the tile's last column meet zeros of W
  for (int l0 = 0; l0 < lend; l0 += kPanel) {
    for (int e = tid; e < kWT * kPanel; e += kWThreads) {
      const int rr = e / kPanel, ll = e - rr * kPanel;
      const int64_t row = row0 + rr;
      xs[rr][ll] = (row < rows && l0 + ll < B.k) ? X[row * B.ldx + l0 + ll] : T(0);
    }
    for (int e = tid; e < kPanel * kWT; e += kWThreads) {
      const int ll = e / kWT, cc = e - ll * kWT;
      const int l = l0 + ll, c = c0 + cc;
      ws[ll][cc] = (l < B.k && c < B.kout && l <= c) ? W[static_cast<int64_t>(B.w0 + l) * a.wld + B.w0 + c] : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int ll = 0; ll < kPanel; ++ll) {
      T u[4], v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        u[q] = xs[ty * 4 + q][ll];
        v[q] = ws[ll][tx * 4 + q];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += u[i] * v[j];
    }
    __syncthreads();
  }
  T* Q = static_cast<T*>(B.Q);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t row = row0 + ty * 4 + i;
    if (row >= rows) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + tx * 4 + j;
      if (c < B.kout) Q[row * B.kout + c] = acc[i][j];
    }
  }
}

// --------------------------------------------------------- grid barrier ----

struct Sync {
  uint32_t* count;
  uint32_t* gen;
  int32_t* status;
  int64_t limit;
};

// Every CTA of the (cooperative) grid arrives; the last one to arrive starts
// the next generation.  The wait is bounded: on expiry the timeout bit is set.
// Returns false once any CTA has recorded a timeout (all CTAs then leave).
__device__ bool grid_sync(const Sync& g) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const uint32_t gen = ld_acquire(g.gen);
    __threadfence();
    if (atomicAdd(g.count, 1u) == gridDim.x - 1) {
      atomicExch(g.count, 0u);
      __threadfence();
      st_release(g.gen, gen + 1);
    } else {
      int64_t i = 0;
      while (ld_acquire(g.gen) == gen) {
        if (++i > g.limit) {
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (!ok) set_status(g.status, kStatusTimeout);
    s_ok = ok && !(ld_acquire(reinterpret_cast<const uint32_t*>(g.status)) & kStatusTimeout);
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ bool timed_out(const int32_t* status) {
  return (*reinterpret_cast<const volatile int32_t*>(status) & kStatusTimeout) != 0;
}

// Waits (bounded) until column blocks b0 and b1 have completed k rounds:
// the CTAs that wrote them in the previous round have published their
// versions (release after the CTA's stores), so a block round waits for its
// two producers only instead of for the whole grid.  Returns false on a
// timeout (the timeout bit is then set) or when another CTA has timed out.
__device__ bool wait_blocks(const uint32_t* ver, int b0, int b1, uint32_t k, const Sync& g) {
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    int ok = 1;
    int64_t i = 0;
    while (ld_acquire(ver + b0) < k || ld_acquire(ver + b1) < k) {
      if (++i > g.limit || (ld_acquire(reinterpret_cast<const uint32_t*>(g.status)) & kStatusTimeout)) {
        ok = 0;
        break;
      }
      __nanosleep(32);
    }
    if (!ok) set_status(g.status, kStatusTimeout);
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ---------------------------------------------------- blocked Cholesky ----

template <typename T>
struct CholSmem {
  T d[kPanel][kPanel + 1];
  T p[kPanel][kPanel + 1];
  T y[kPanel];
};

// In-place semi-definite Cholesky (upper, A = R^T R) of the n x n row-major
// A in global memory.  diag0: the diagonal A started with; act: columns
// marked 0 stay dependent; y: 1 / R_kk (0 for a dependent column).  Right-
// looking by 32-column panels: factor the diagonal block (CTA 0), solve the
// panel's rows to the right (all CTAs, a column each), update the trailing
// upper triangle (all CTAs, 32 x 32 tiles).
template <typename T>
__device__ bool chol_blocked(T* A, int n, const T* diag0, int32_t* act, T* y, T tol, const Sync& sync,
                             CholSmem<T>& sm) {
  const int tid = threadIdx.x;
  for (int k0 = 0; k0 < n; k0 += kPanel) {
    const int kb = n - k0 < kPanel ? n - k0 : kPanel;
    const int k1 = k0 + kb;
    if (blockIdx.x == 0) {
      for (int e = tid; e < kPanel * kPanel; e += blockDim.x) {
        const int r = e / kPanel, c = e % kPanel;
        sm.d[r][c] = (r < kb && c < kb && c >= r) ? A[static_cast<int64_t>(k0 + r) * n + k0 + c] : T(0);
      }
      __syncthreads();
      for (int j = 0; j < kb; ++j) {
        const int col = k0 + j;
        const T d = sm.d[j][j];
        const int was = act[col];
        int ok = was;
        if (!isfinite(d)) ok = 0;
        if (!(d > tol * diag0[col]) || !(diag0[col] > T(0))) ok = 0;
        const bool dropped = was && !ok && isfinite(d) && diag0[col] > T(0);
        const T yj = ok ? rsqrt_pivot(d) : T(0);
        __syncthreads();  // every thread has read the pivot
        if (tid >= j && tid < kb) sm.d[j][tid] *= yj;
        if (tid == 0) {
          if (!isfinite(d)) set_status(sync.status, kStatusNotSpd);
          if (dropped) note_dropped(sync.status, col);
          act[col] = ok;
          y[col] = yj;
          sm.y[j] = yj;
        }
        __syncthreads();
        for (int e = tid; e < kb * kb; e += blockDim.x) {
          const int i = e / kb, c = e % kb;
          if (i > j && c >= i) sm.d[i][c] -= sm.d[j][i] * sm.d[j][c];
        }
        __syncthreads();
      }
      for (int e = tid; e < kb * kb; e += blockDim.x) {
        const int r = e / kb, c = e % kb;
        if (c >= r) A[static_cast<int64_t>(k0 + r) * n + k0 + c] = sm.d[r][c];
      }
    }
    if (!grid_sync(sync)) return false;
    if (k1 >= n) break;
    // panel rows right of the diagonal block: R[j][c] = (A[j][c] - sum_{i<j} R[i][j] R[i][c]) / R[j][j]
    for (int e = tid; e < kPanel * kPanel; e += blockDim.x) {
      const int r = e / kPanel, c = e % kPanel;
      sm.d[r][c] = (r < kb && c < kb && c >= r) ? A[static_cast<int64_t>(k0 + r) * n + k0 + c] : T(0);
    }
    if (tid < kPanel) sm.y[tid] = tid < kb ? y[k0 + tid] : T(0);
    __syncthreads();
    for (int c = k1 + blockIdx.x * blockDim.x + tid; c < n; c += gridDim.x * blockDim.x) {
      T v[kPanel];
#pragma unroll
      for (int j = 0; j < kPanel; ++j) {
        if (j < kb) {
          T s = A[static_cast<int64_t>(k0 + j) * n + c];
#pragma unroll
          for (int i = 0; i < j; ++i) s -= sm.d[i][j] * v[i];
          v[j] = s * sm.y[j];
          A[static_cast<int64_t>(k0 + j) * n + c] = v[j];
        } else {
          v[j] = T(0);
        }
      }
    }
    if (!grid_sync(sync)) return false;
    // trailing update of the upper triangle of A[k1:, k1:]
    const int nt = (n - k1 + kPanel - 1) / kPanel;
    const int ntt = nt * (nt + 1) / 2;
    for (int t = blockIdx.x; t < ntt; t += gridDim.x) {
      int ti, tj;
      upper_tile(t, nt, ti, tj);
      const int i0 = k1 + ti * kPanel, c0 = k1 + tj * kPanel;
      for (int e = tid; e < kPanel * kPanel; e += blockDim.x) {
        const int j = e / kPanel, q = e % kPanel;
        sm.d[j][q] = (j < kb && i0 + q < n) ? A[static_cast<int64_t>(k0 + j) * n + i0 + q] : T(0);
        sm.p[j][q] = (j < kb && c0 + q < n) ? A[static_cast<int64_t>(k0 + j) * n + c0 + q] : T(0);
      }
      __syncthreads();
      for (int e = tid; e < kPanel * kPanel; e += blockDim.x) {
        const int ii = e / kPanel, cc = e % kPanel;
        const int i = i0 + ii, c = c0 + cc;
        if (i < n && c < n && c >= i) {
          T s0 = T(0), s1 = T(0);
#pragma unroll
          for (int j = 0; j < kPanel; j += 2) {
            s0 += sm.d[j][ii] * sm.p[j][cc];
            s1 += sm.d[j + 1][ii] * sm.p[j + 1][cc];
          }
          A[static_cast<int64_t>(i) * n + c] -= s0 + s1;
        }
      }
      __syncthreads();
    }
    if (!grid_sync(sync)) return false;
  }
  return true;
}

// W = R^{-1} on the independent columns (R upper in A), one column per warp:
// W[j][j] = 1 / R[j][j], W[i][j] = -(sum_{k=i+1..j} R[i][k] W[k][j]) / R[i][i].
template <typename T>
__device__ void inverse_columns(const T* A, T* Wt, int n, const int32_t* act, T* wcol) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T* w = wcol + warp * n;
  for (int j = blockIdx.x * nw + warp; j < n; j += gridDim.x * nw) {
    if (act[j]) {
      if (lane == 0) w[j] = T(1) / A[static_cast<int64_t>(j) * n + j];
      __syncwarp();
      for (int i = j - 1; i >= 0; --i) {
        if (!act[i]) {
          if (lane == 0) w[i] = T(0);
          __syncwarp();
          continue;
        }
        const T* Ri = A + static_cast<int64_t>(i) * n;
        T s = T(0);
        for (int k = i + 1 + lane; k <= j; k += 32) s += Ri[k] * w[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) w[i] = -s / Ri[i];
        __syncwarp();
      }
    }
    for (int i = lane; i < n; i += 32) Wt[static_cast<int64_t>(i) * n + j] = (act[j] && i <= j) ? w[i] : T(0);
    __syncwarp();
  }
}

struct DenseArgs {
  int n;
  double tol;
  const double* G;     // G1 or G2
  void* A;             // n x n compute type
  void* Tw;            // n x n compute type
  void* y;
  void* d0;
  int32_t* active;
  double* R1;
  double* W;
  float* Wf;
  double* E;           // n x n FP64 scratch
  double* X;           // n x n FP64
  double* R;
  double* R_out;
  int64_t ldr;
  int refine;
  double shift_rel;    // shifted CholeskyQR3: relative shift of the first factorisation
  int from_r;          // first factorisation: G holds the upper-triangular R to invert
  DevHeader* h;
  int64_t spin_limit;
};

__device__ __forceinline__ Sync make_sync(const DenseArgs& a) {
  return Sync{&a.h->bar_count, &a.h->bar_gen, &a.h->status, a.spin_limit};
}

template <typename T>
__global__ void __launch_bounds__(kWThreads) wide_chol_first_kernel(DenseArgs a) {
  pdl_enter();
  __shared__ CholSmem<T> sm;
  extern __shared__ __align__(16) unsigned char wcol_raw[];
  if (timed_out(&a.h->status)) return;
  const Sync sync = make_sync(a);
  const int n = a.n;
  T* A = static_cast<T*>(a.A);
  T* Wt = static_cast<T*>(a.Tw);
  T* y = static_cast<T*>(a.y);
  T* d0 = static_cast<T*>(a.d0);
  const int64_t nn = static_cast<int64_t>(n) * n;
  const int64_t gt = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x, gs = static_cast<int64_t>(gridDim.x) * blockDim.x;
  // shifted CholeskyQR3: shift_rel trace(G) on the non-zero diagonal entries
  double shift = 0.0;
  if (a.shift_rel > 0.0 && !a.from_r) {
    for (int k = 0; k < n; ++k) shift += a.G[static_cast<int64_t>(k) * n + k];
    shift *= a.shift_rel;
  }
  for (int64_t e = gt; e < nn; e += gs) {
    const int64_t i = e / n, j = e - i * n;
    const double g = a.G[e];
    A[e] = static_cast<T>(i == j && g > 0.0 ? g + shift : g);
  }
  for (int64_t k = gt; k < n; k += gs) {
    const double g = a.G[k * n + k];
    d0[k] = static_cast<T>(g > 0.0 ? g + shift : g);
    a.active[k] = a.from_r ? (g != 0.0) : 1;
  }
  if (!grid_sync(sync)) return;
  // from_r: G is the upper-triangular R of the previous pass, inverted as is
  if (!a.from_r && !chol_blocked<T>(A, n, d0, a.active, y, static_cast<T>(a.tol), sync, sm)) return;
  inverse_columns<T>(A, Wt, n, a.active, reinterpret_cast<T*>(wcol_raw));
  if (!grid_sync(sync)) return;
  for (int64_t e = gt; e < nn; e += gs) {
    const int i = static_cast<int>(e / n), j = static_cast<int>(e - static_cast<int64_t>(i) * n);
    a.R1[e] = (j >= i && a.active[i]) ? (a.from_r ? a.G[e] : static_cast<double>(A[e])) : 0.0;
    // dependent columns pass through the second pass unchanged (identity)
    double w = (j >= i) ? static_cast<double>(Wt[e]) : 0.0;
    if (i == j && !a.active[i]) w = 1.0;
    if (sizeof(T) == 4) {  // a value both the SIMT and tensor-core engines use exactly (hi + lo in TF32)
      const float v = static_cast<float>(w);
      const float hv = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
      const float lv = __uint_as_float((__float_as_uint(v - hv) + 0x1000u) & 0xFFFFE000u);
      w = static_cast<double>(hv + lv);
    }
    a.W[e] = w;
    a.Wf[e] = static_cast<float>(w);
  }
}

// sum_{k=i..j} A[i][k] B[k][j] of two upper-triangular n x n matrices, FP64.
template <typename TA, typename TB>
__device__ __forceinline__ double upper_dot_n(const TA* A, const TB* B, int n, int i, int j) {
  double s0 = 0.0, s1 = 0.0;
  int k = i;
  const TA* Ai = A + static_cast<int64_t>(i) * n;
  for (; k + 1 <= j; k += 2) {
    s0 += static_cast<double>(Ai[k]) * static_cast<double>(B[static_cast<int64_t>(k) * n + j]);
    s1 += static_cast<double>(Ai[k + 1]) * static_cast<double>(B[static_cast<int64_t>(k + 1) * n + j]);
  }
  if (k <= j) s0 += static_cast<double>(Ai[k]) * static_cast<double>(B[static_cast<int64_t>(k) * n + j]);
  return s0 + s1;
}

template <typename T>
__global__ void __launch_bounds__(kWThreads) wide_chol_second_kernel(DenseArgs a) {
  pdl_enter();
  __shared__ CholSmem<T> sm;
  if (timed_out(&a.h->status)) return;
  const Sync sync = make_sync(a);
  const int n = a.n;
  T* A = static_cast<T*>(a.A);
  T* y = static_cast<T*>(a.y);
  T* d0 = static_cast<T*>(a.d0);
  int32_t* act = a.active;
  const int64_t nn = static_cast<int64_t>(n) * n;
  const int64_t gt = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x, gs = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t e = gt; e < nn; e += gs) A[e] = static_cast<T>(a.G[e]);
  for (int64_t k = gt; k < n; k += gs) d0[k] = static_cast<T>(a.G[k * n + k]);
  if (a.refine) {
    // E = I - W R1 on the independent block
    for (int64_t e = gt; e < nn; e += gs) {
      const int i = static_cast<int>(e / n), j = static_cast<int>(e - static_cast<int64_t>(i) * n);
      a.E[e] = (j >= i && act[i] && act[j]) ? (i == j ? 1.0 : 0.0) - upper_dot_n(a.W, a.R1, n, i, j) : 0.0;
    }
    if (!grid_sync(sync)) return;
  }
  // X = W^{-1}: R1 + R1 E (refined) or R1, identity on the dependent columns
  for (int64_t e = gt; e < nn; e += gs) {
    const int i = static_cast<int>(e / n), j = static_cast<int>(e - static_cast<int64_t>(i) * n);
    double x = 0.0;
    if (j >= i && act[i] && act[j]) x = a.R1[e] + (a.refine ? upper_dot_n(a.R1, a.E, n, i, j) : 0.0);
    if (i == j && !act[i]) x = 1.0;
    a.X[e] = x;
  }
  if (!grid_sync(sync)) return;
  if (!chol_blocked<T>(A, n, d0, act, y, static_cast<T>(a.tol), sync, sm)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    int dep = 0;
    for (int k = 0; k < n; ++k) dep += act[k] ? 0 : 1;
    a.h->dep_cols = dep;
  }
  // R = R2 X in FP64; rows of dependent columns are zero
  for (int64_t e = gt; e < nn; e += gs) {
    const int i = static_cast<int>(e / n), j = static_cast<int>(e - static_cast<int64_t>(i) * n);
    const double s = (j >= i && act[i]) ? upper_dot_n(A, a.X, n, i, j) : 0.0;
    a.R[e] = s;
    if (a.R_out) a.R_out[static_cast<int64_t>(i) * a.ldr + j] = s;
  }
}

// ------------------------------------------------------------- Jacobi ----

struct JacArgs {
  const double* R;
  int64_t ldr;
  int n;
  int nblk;         // blocks of JW columns (even; the padding columns are zero)
  int max_sweeps;
  double tol;
  void* U;          // column-major, nblk * JW columns of n rows
  void* V;
  DevHeader* h;
  int64_t spin_limit;
};

__device__ __forceinline__ void jac_rotation(float al, float be, float ga, float& c, float& s) {
  const float z = __fdividef(be - al, 2.f * ga);
  const float az = fabsf(z);
  const float q = 1.f + z * z;
  const float t = az > 1e18f ? __fdividef(0.5f, z) : copysignf(__fdividef(1.f, az + q * rsqrtf(q)), z);
  c = rsqrtf(1.f + t * t);
  s = c * t;
}
__device__ __forceinline__ void jac_rotation(double al, double be, double ga, double& c, double& s) {
  const double z = (be - al) / (2.0 * ga);
  const double t = (z >= 0.0 ? 1.0 : -1.0) / (fabs(z) + sqrt(1.0 + z * z));
  c = 1.0 / sqrt(1.0 + t * t);
  s = c * t;
}

__device__ __forceinline__ void rr_pair(int round, int g, int m, int& p, int& q) {
  // round-robin tournament over m (even) players: m - 1 rounds of m / 2 games
  p = g == 0 ? round : (round + g) % (m - 1);
  q = g == 0 ? m - 1 : (round - g + (m - 1)) % (m - 1);
  if (p > q) {
    const int t = p;
    p = q;
    q = t;
  }
}

// Four consecutive shared-memory entries (16-byte aligned).
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
  const double2 q0 = reinterpret_cast<const double2*>(p)[0], q1 = reinterpret_cast<const double2*>(p)[1];
  v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
}

// JW: block width in columns; a CTA of JW warps works on a pair of blocks,
// W2 = 2 JW columns of U (and V).  A block round (Section 3's one-sided
// Jacobi, by blocks): the pair's columns are staged in shared memory
// (column-major, column stride n + 1), their Gram G = S^T S is formed by
// 4 x 4 register tiles over row splits (fixed reduction order, so G is
// exactly symmetric), one cyclic sweep of two-sided rotations runs on G
// (in each of the W2 - 1 inner rounds every lane forms the rotation of its
// column pair and warp w writes rows p, q of J^T G J, from the previous
// buffer, and of Q J: one barrier per inner round; the sweep is skipped
// when no pair of G passes the rotation test), and U <- S Q and V <- V Q
// are written back only when a rotation was applied.  Between rounds a CTA
// waits for the two CTAs that wrote its blocks (per-block round counters);
// the grid meets once per sweep to complete the convergence flag.  An inner
// round thus touches the W2 x W2 entries of G and Q instead of the 2 n W2
// entries of the n-row columns of U and V; the rotation test is the column
// test |g_pq| > tol sqrt(g_pp g_qq) on G.  (FP32 dot products and rotations
// keep their accuracy relative to sqrt(g_pp g_qq) under column scaling, so
// graded columns converge as in the column form.)
template <typename T, bool kWithV, int JW>
__global__ void __launch_bounds__(32 * JW) wide_jacobi_kernel(JacArgs a) {
  pdl_enter();
  constexpr int W2 = 2 * JW;
  constexpr int NT = 32 * JW;
  constexpr int TD = W2 / 4;       // 4 x 4 tiles per dimension of G
  constexpr int NTI = TD * TD;
  constexpr int KS = NT / NTI;     // row splits of the Gram
  constexpr int LG = W2 + 1;       // row stride of G
  constexpr int kRowsPer = (kMaxWideWidth + NT - 1) / NT;  // rows of S staged per thread
  static_assert(W2 % 4 == 0 && NT % NTI == 0 && W2 <= 32, "block shape");
  extern __shared__ __align__(16) unsigned char jsm[];
  const int n = a.n;
  const int ls = n + 1;                                          // column stride of S
  T* S = reinterpret_cast<T*>(jsm);                              // W2 columns of n rows
  T* Pg = S + static_cast<int64_t>(W2) * ls;                     // KS partial Grams
  T* G = Pg + KS * W2 * W2;                                      // two W2 x LG buffers
  T* Qm = G + 2 * W2 * LG;                                       // W2 x W2
  __shared__ int s_conv;
  if (timed_out(&a.h->status)) return;
  const Sync sync{&a.h->bar_count, &a.h->bar_gen, &a.h->status, a.spin_limit};
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int np = a.nblk * JW;
  T* U = static_cast<T*>(a.U);
  T* V = static_cast<T*>(a.V);
  const int64_t gt = static_cast<int64_t>(blockIdx.x) * blockDim.x + tid, gs = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t e = gt; e < static_cast<int64_t>(np) * n; e += gs) {
    const int c = static_cast<int>(e / n), r = static_cast<int>(e - static_cast<int64_t>(c) * n);
    U[e] = c < n ? static_cast<T>(a.R[static_cast<int64_t>(r) * a.ldr + c]) : T(0);
    if (kWithV) V[e] = (c == r) ? T(1) : T(0);
  }
  if (blockIdx.x == 0 && tid == 0) {
    a.h->sweep_any[0] = 0u;
    a.h->sweep_any[1] = 0u;
    a.h->sweep_any[2] = 0u;
  }
  uint32_t* ver = a.h->blk_ver;
  if (gt < a.nblk) ver[gt] = 0u;
  // ||R||_F^2, the same sum in every CTA
  __shared__ double s_part[JW];
  double f = 0.0;
  for (int64_t e0 = tid; e0 < static_cast<int64_t>(n) * n; e0 += 8 * NT) {  // 8 loads in flight per thread
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t e = e0 + static_cast<int64_t>(u) * NT;
      const int r = static_cast<int>(e / n), c = static_cast<int>(e - static_cast<int64_t>(r) * n);
      v[u] = e < static_cast<int64_t>(n) * n ? static_cast<double>(static_cast<T>(a.R[static_cast<int64_t>(r) * a.ldr + c]))
                                             : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) f += v[u] * v[u];
  }
  for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
  if (lane == 0) s_part[warp] = f;
  if (!grid_sync(sync)) return;
  double fro = 0.0;
  for (int w = 0; w < JW; ++w) fro += s_part[w];
  // columns below n eps64 ||R||_F are rounding noise of a rank-deficient R
  // and take no part in rotations (the FP64 unit even for FP32 sweeps: FP32
  // dot products keep their relative accuracy under column scaling, so
  // legitimately small columns of a graded R must keep rotating)
  const double eps64 = 1.1102230246251565e-16;
  const T negligible = static_cast<T>((n * eps64) * (n * eps64) * fro);
  const T tol2 = static_cast<T>(a.tol) * static_cast<T>(a.tol);
  const int pairs = a.nblk / 2;
  // Gram tile of this thread: rows [r0, r1) of split ks, entries (4 ti + u, 4 tj + v)
  const int ks = tid / NTI, ti = (tid % NTI) / TD, tj = tid % TD;
  const int rs = (n + KS - 1) / KS;
  const int r0 = ks * rs < n ? ks * rs : n, r1 = r0 + rs < n ? r0 + rs : n;
  int sweep = 0;
  bool converged = false;
  for (; sweep < a.max_sweeps; ++sweep) {
    if (blockIdx.x == 0 && tid == 0) atomicExch(&a.h->sweep_any[(sweep + 1) % 3], 0u);
    for (int round = 0; round < a.nblk - 1; ++round) {
      const uint32_t K = static_cast<uint32_t>(sweep * (a.nblk - 1) + round);  // rounds before this one
      for (int g = blockIdx.x; g < pairs; g += gridDim.x) {
        int bp, bq;
        rr_pair(round, g, a.nblk, bp, bq);
        if (!wait_blocks(ver, bp, bq, K, sync)) return;
        auto col_of = [&](int lc) { return lc < JW ? bp * JW + lc : bq * JW + lc - JW; };
        // staging: every load of the thread is issued before its stores (one memory round trip)
        {
          T x[kRowsPer][W2];
#pragma unroll
          for (int h = 0; h < kRowsPer; ++h) {
            const int r = tid + h * NT;
#pragma unroll
            for (int lc = 0; lc < W2; ++lc) x[h][lc] = r < n ? U[static_cast<int64_t>(col_of(lc)) * n + r] : T(0);
          }
#pragma unroll
          for (int h = 0; h < kRowsPer; ++h) {
            const int r = tid + h * NT;
            if (r < n) {
#pragma unroll
              for (int lc = 0; lc < W2; ++lc) S[lc * ls + r] = x[h][lc];
            }
          }
        }
        for (int e = tid; e < W2 * W2; e += NT) Qm[e] = (e / W2 == e % W2) ? T(1) : T(0);
        __syncthreads();
        {
          T acc[4][4];
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
          const T* si = S + (4 * ti) * ls;
          const T* sj = S + (4 * tj) * ls;
          for (int r = r0; r < r1; ++r) {
            T x[4], y[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              x[u] = si[u * ls + r];
              y[u] = sj[u * ls + r];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int v = 0; v < 4; ++v) acc[u][v] = fma(x[u], y[v], acc[u][v]);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) Pg[(ks * W2 + 4 * ti + u) * W2 + 4 * tj + v] = acc[u][v];
        }
        __syncthreads();
        for (int e = tid; e < W2 * W2; e += NT) {
          T s_ = T(0);
          for (int k = 0; k < KS; ++k) s_ += Pg[k * W2 * W2 + e];
          G[(e / W2) * LG + e % W2] = s_;
        }
        __syncthreads();
        // inner sweep on G, double-buffered, one barrier per inner round: lane
        // j forms the rotation of its own column pair (j, j') and warp w the
        // rows p, q of its pair of G' = J^T G J (and of Q J) from the previous
        // G.  With (c, s) the pair's rotation and sg_j = -s for the lower
        // column, +s for the upper: (G J)[k][j] = c G[k][j] + sg_j G[k][j'].
        // no pair of the block passes the rotation test: the sweep would leave G unchanged
        int need = 0;
        for (int e = tid; e < W2 * W2; e += NT) {
          const int i = e / W2, j = e % W2;
          if (i < j) {
            const T al = G[i * LG + i], be = G[j * LG + j], ga = G[i * LG + j];
            need |= (al > negligible && be > negligible && ga * ga > tol2 * al * be) ? 1 : 0;
          }
        }
        need = __syncthreads_or(need);
        int any = 0;
        T* Gc = G;
        T* Gn = G + W2 * LG;
        constexpr int M1 = W2 - 1;
        // the first IW warps run the inner sweep, PPW pairs each per inner
        // round, and meet at a barrier of their own (a barrier of all the
        // CTA's warps per inner round cost more than the round's work)
        constexpr int IW = JW < 4 ? JW : 4;
        constexpr int PPW = (W2 / 2) / IW;
        static_assert(IW * PPW == W2 / 2, "inner sweep split");
        if (warp < IW) {
          for (int ir = 0; need && ir < M1; ++ir) {
            const int j = lane < W2 ? lane : 0;  // lanes beyond W2 mirror lane 0 and store nothing
            int jp = (2 * ir - j) % M1;
            jp += jp < 0 ? M1 : 0;
            jp = j == ir ? M1 : jp;
            jp = j == M1 ? ir : jp;
            const int lo = j < jp ? j : jp, hi = j < jp ? jp : j;
            const T al = Gc[lo * LG + lo], be = Gc[hi * LG + hi], ga = Gc[lo * LG + hi];
            const bool rot = al > negligible && be > negligible && ga * ga > tol2 * al * be;
            T c = T(1), s = T(0);
            if (rot) jac_rotation(al, be, ga, c, s);
            const T sg = j < jp ? -s : s;
            int pp[PPW], qq[PPW];
            T gp[PPW], gq[PPW], qp[PPW], qqv[PPW];
#pragma unroll
            for (int t = 0; t < PPW; ++t) {
              rr_pair(ir, warp + t * IW, W2, pp[t], qq[t]);
              const int p = pp[t], q = qq[t];
              const T gpj = Gc[p * LG + j], gpjp = Gc[p * LG + jp], gqj = Gc[q * LG + j], gqjp = Gc[q * LG + jp];
              const T qpj = Qm[p * W2 + j], qpjp = Qm[p * W2 + jp], qqj = Qm[q * W2 + j], qqjp = Qm[q * W2 + jp];
              const T cw = __shfl_sync(0xffffffffu, c, p), sw = __shfl_sync(0xffffffffu, s, p);  // the pair (p, q)
              const T hp = c * gpj + sg * gpjp, hq = c * gqj + sg * gqjp;
              gp[t] = cw * hp - sw * hq;
              gq[t] = sw * hp + cw * hq;
              qp[t] = c * qpj + sg * qpjp;
              qqv[t] = c * qqj + sg * qqjp;
            }
            __syncwarp();  // rows p, q of Q are read above by the lanes that own their partners
            if (lane < W2) {
#pragma unroll
              for (int t = 0; t < PPW; ++t) {
                Gn[pp[t] * LG + j] = gp[t];
                Gn[qq[t] * LG + j] = gq[t];
                Qm[pp[t] * W2 + j] = qp[t];
                Qm[qq[t] * W2 + j] = qqv[t];
              }
            }
            any |= rot ? 1 : 0;
            asm volatile("bar.sync 2, %0;" ::"n"(32 * IW) : "memory");
            T* t_ = Gc;
            Gc = Gn;
            Gn = t_;
          }
        }
        any = __syncthreads_or(any);
        if (any) {
          // U <- S Q and V <- V Q, one row per thread (coalesced in the column-major U and V)
          // (Q read four entries at a time: broadcast loads shared by the warp)
          auto times_q = [&](const T (&x)[W2], T* dst, int r) {
#pragma unroll 2
            for (int j4 = 0; j4 < W2; j4 += 4) {
              T o[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
              for (int k = 0; k < W2; ++k) {
                T qv[4];
                ld4(Qm + k * W2 + j4, qv);
#pragma unroll
                for (int v = 0; v < 4; ++v) o[v] = fma(x[k], qv[v], o[v]);
              }
#pragma unroll
              for (int v = 0; v < 4; ++v) dst[static_cast<int64_t>(col_of(j4 + v)) * n + r] = o[v];
            }
          };
          for (int r = tid; r < n; r += NT) {
            T x[W2];
#pragma unroll
            for (int k = 0; k < W2; ++k) x[k] = S[k * ls + r];
            times_q(x, U, r);
            if (kWithV) {
#pragma unroll
              for (int k = 0; k < W2; ++k) x[k] = V[static_cast<int64_t>(col_of(k)) * n + r];
              times_q(x, V, r);
            }
          }
          if (tid == 0) atomicOr(&a.h->sweep_any[sweep % 3], 1u);
        }
        __syncthreads();  // every store of the CTA is issued
        if (tid == 0) {
          __threadfence();
          st_release(ver + bp, K + 1);
          st_release(ver + bq, K + 1);
        }
      }
    }
    if (!grid_sync(sync)) return;  // the sweep's flag is complete
    if (tid == 0) s_conv = ld_acquire(&a.h->sweep_any[sweep % 3]) == 0u;
    __syncthreads();
    if (s_conv) {
      converged = true;
      ++sweep;
      break;
    }
  }
  if (blockIdx.x == 0 && tid == 0) {
    if (!converged) set_status(&a.h->status, kStatusNoConvergence);
    a.h->jacobi_sweeps = sweep;
  }
}

// sigma_j (unsorted).  Plain path: ||u_j|| in FP64.  Mixed path: the FP64
// Rayleigh quotient ||R v_j|| / ||v_j||, whose error is second order in the
// FP32 error of v_j, d sigma ~ (delta sigma_max)^2 / (2 sigma_j) -- small for
// the large values, but of order delta sigma_max for sigma_j near zero; the
// FP32 column norm ||u_j|| has an absolute error of a few FP32 ulps of
// sigma_max (and keeps relative accuracy under column scaling), so it is
// kept too and wide_sort_kernel takes it for sigma_j < 1e-3 max_k ||u_k||.
// One CTA per column, one warp per row of R.
template <typename T, bool kWithV>
__global__ void __launch_bounds__(kWThreads) wide_sigma_kernel(const double* R, int64_t ldr, int n, const T* U,
                                                               const T* V, double* sig, double* unorm,
                                                               const int32_t* status) {
  pdl_enter();
  __shared__ double vj[kMaxWideWidth];
  __shared__ double red[kWThreads / 32], redu[kWThreads / 32];
  if (timed_out(status)) return;
  const int j = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double acc = 0.0, uacc = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const double u = static_cast<double>(U[static_cast<int64_t>(j) * n + k]);
    uacc += u * u;
  }
  for (int o = 16; o > 0; o >>= 1) uacc += __shfl_xor_sync(0xffffffffu, uacc, o);
  if (kWithV) {
    for (int k = threadIdx.x; k < n; k += blockDim.x) vj[k] = static_cast<double>(V[static_cast<int64_t>(j) * n + k]);
    __syncthreads();
    for (int i = warp; i < n; i += kWThreads / 32) {
      const double* Ri = R + static_cast<int64_t>(i) * ldr;
      double s = 0.0;
      for (int k = i + lane; k < n; k += 32) s += Ri[k] * vj[k];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) acc += s * s;
    }
  }
  if (lane == 0) {
    red[warp] = acc;
    redu[warp] = uacc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double num = 0.0, un = 0.0;
    for (int w = 0; w < kWThreads / 32; ++w) {
      num += red[w];
      un += redu[w];
    }
    unorm[j] = sqrt(un);
    if (kWithV) {
      double den = 0.0;
      for (int k = 0; k < n; ++k) den += vj[k] * vj[k];
      sig[j] = den > 0.0 ? sqrt(num / den) : 0.0;
    } else {
      sig[j] = sqrt(un);
    }
  }
}

__global__ void __launch_bounds__(kMaxWideWidth) wide_sort_kernel(const double* sig, const double* unorm, int n,
                                                                 double* sigma, const int32_t* status) {
  pdl_enter();
  __shared__ double s_val[kMaxWideWidth];
  __shared__ double s_max;
  if (timed_out(status)) return;
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int k = 0; k < n; ++k) m = unorm[k] > m ? unorm[k] : m;
    s_max = m;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) s_val[j] = unorm[j] < 1e-3 * s_max ? unorm[j] : sig[j];
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double v = s_val[j];
    int rank = 0;
    for (int k = 0; k < n; ++k) {
      const double w = s_val[k];
      rank += (w > v) || (w == v && k < j);
    }
    sigma[rank] = v;
  }
}

// sigma descending and, for each value, its right singular vector: column
// j of V (n x n row-major, leading dimension ldv) is the unit-norm column of
// the accumulated rotations that belongs to sigma_j, its sign chosen so that
// its largest-magnitude component is positive.  One CTA.
template <typename T>
__global__ void __launch_bounds__(kMaxWideWidth) wide_sort_v_kernel(const double* sig, const double* unorm, int n,
                                                                   const T* V, double* sigma, double* V_out,
                                                                   int64_t ldv, const int32_t* status) {
  pdl_enter();
  __shared__ double s_val[kMaxWideWidth], s_scale[kMaxWideWidth];
  __shared__ int s_rank[kMaxWideWidth];
  __shared__ double s_max;
  if (timed_out(status)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int k = 0; k < n; ++k) m = unorm[k] > m ? unorm[k] : m;
    s_max = m;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) s_val[j] = unorm[j] < 1e-3 * s_max ? unorm[j] : sig[j];
  // per column: 1 / ||v_j|| times the sign of its largest-magnitude entry
  for (int j = warp; j < n; j += nw) {
    const T* vj = V + static_cast<int64_t>(j) * n;
    double ss = 0.0, big = 0.0;
    int at = 0;
    for (int i = lane; i < n; i += 32) {
      const double v = static_cast<double>(vj[i]);
      ss += v * v;
      if (fabs(v) > fabs(big)) {
        big = v;
        at = i;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      ss += __shfl_xor_sync(0xffffffffu, ss, o);
      const double ob = __shfl_xor_sync(0xffffffffu, big, o);
      const int oa = __shfl_xor_sync(0xffffffffu, at, o);
      if (fabs(ob) > fabs(big) || (fabs(ob) == fabs(big) && oa < at)) {
        big = ob;
        at = oa;
      }
    }
    if (lane == 0) s_scale[j] = ss > 0.0 ? (big < 0.0 ? -1.0 : 1.0) / sqrt(ss) : 0.0;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double v = s_val[j];
    int rank = 0;
    for (int k = 0; k < n; ++k) {
      const double w = s_val[k];
      rank += (w > v) || (w == v && k < j);
    }
    s_rank[j] = rank;
    sigma[rank] = v;
  }
  __syncthreads();
  for (int64_t e = threadIdx.x; e < static_cast<int64_t>(n) * n; e += blockDim.x) {
    const int j = static_cast<int>(e / n), i = static_cast<int>(e - static_cast<int64_t>(j) * n);
    V_out[static_cast<int64_t>(i) * ldv + s_rank[j]] = static_cast<double>(V[e]) * s_scale[j];
  }
}

// ---------------------------------------------------------- host side ----

// Jobs of each block's Gram.  tc_mask bit i: block i (0 head, 1 A tails,
// 2 B tails) runs on the tensor cores.  CUDA-core jobs come first in the
// partial buffer (64 x 64 doubles each), tensor-core jobs after them
// (128 x 128 each); *part_doubles is the buffer's size.
void wide_geometry(int pass, int64_t m1, int n1, int64_t m2, int n2, int num_sms, int tc_mask, WideBlock b[3],
                   int* gram_jobs, int* form_jobs, int* tc_jobs, int64_t* part_doubles) {
  const int n = n1 + n2;
  const int64_t rows[3] = {m1, m1, m2};
  const int ks[3] = {n, n1, n2};
  const int kouts[3] = {n, pass == 1 ? n1 : n, n2};
  const int offs[3] = {0, 0, n1};
  const int w0s[3] = {0, 0, n1};
  int gj = 0, fj = 0, tj = 0;
  for (int i = 0; i < 3; ++i) {
    WideBlock& B = b[i];
    B = WideBlock{};
    B.k = ks[i];
    B.kout = kouts[i];
    B.off = offs[i];
    B.w0 = w0s[i];
    B.rows = rows[i];
    B.tc = (tc_mask >> i) & 1;
    B.tiles = (B.kout + kWT - 1) / kWT;  // (also the formation's column tiles)
    if (!B.tc) {
      B.ntiles = B.tiles * (B.tiles + 1) / 2;
      const int64_t target = 4 * static_cast<int64_t>(num_sms) / B.ntiles;
      int64_t splits = (B.rows + 1023) / 1024;
      if (splits > target) splits = target;
      if (splits < 1) splits = 1;
      int64_t sr = (B.rows + splits - 1) / splits;
      sr = (sr + kWRows - 1) / kWRows * kWRows;
      if (sr < kWRows) sr = kWRows;
      B.split_rows = sr;
      B.splits = B.rows > 0 ? static_cast<int>((B.rows + sr - 1) / sr) : 0;
      B.job0 = gj;
      B.njobs = B.ntiles * B.splits;
      gj += B.njobs;
      B.tw = kWT;
      B.rtiles = B.tiles;
      B.rsplits = B.splits;
    } else {
      B.tc_tiles = (B.kout + kWideTcTile - 1) / kWideTcTile;
      const int nt = B.tc_tiles * (B.tc_tiles + 1) / 2;
      int64_t target = 2 * static_cast<int64_t>(num_sms) / nt;
      if (target < 1) target = 1;
      int64_t splits = (B.rows + 1023) / 1024;
      if (splits > target) splits = target;
      if (splits < 1) splits = 1;
      int64_t sr = (B.rows + splits - 1) / splits;
      sr = (sr + 63) / 64 * 64;  // whole drains of 64 rows
      B.tc_split_rows = sr;
      B.tc_splits = B.rows > 0 ? static_cast<int>((B.rows + sr - 1) / sr) : 0;
      B.tc_njobs = nt * B.tc_splits;
      B.tw = kWideTcTile;
      B.rtiles = B.tc_tiles;
      B.rsplits = B.tc_splits;
    }
    B.fjob0 = fj;
    B.fjobs = pass == 2 && B.rows > 0 ? static_cast<int>((B.rows + kWT - 1) / kWT) * B.tiles : 0;
    fj += B.fjobs;
  }
  int64_t pb = static_cast<int64_t>(gj) * kWT * kWT;
  for (int i = 0; i < 3; ++i) {
    WideBlock& B = b[i];
    if (!B.tc) {
      B.pbase = static_cast<int64_t>(B.job0) * kWT * kWT;
    } else {
      B.pbase = pb;
      pb += static_cast<int64_t>(B.tc_njobs) * kWideTcTile * kWideTcTile;
      tj += B.tc_njobs;
    }
  }
  *gram_jobs = gj;
  *form_jobs = fj;
  *tc_jobs = tj;
  *part_doubles = pb;
}

double wide_tol(const Plan& p) { return p.rank_tol > 0 ? p.rank_tol : (p.mixed ? 1e-5 : 1e-13); }

template <typename K, typename... Args>
cudaError_t launch_cooperative(K kern, int grid, int block, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

DenseArgs dense_args(const Plan& p, int second, double* R_out, int64_t ldr) {
  DenseArgs a{};
  a.n = p.n;
  a.tol = wide_tol(p);
  a.G = second ? p.G2 : p.G1;
  a.A = p.Aw;
  a.Tw = p.Tw;
  a.y = p.yw;
  a.d0 = p.d0w;
  a.active = p.active;
  a.R1 = p.R1;
  a.W = p.W;
  a.Wf = p.Wf;
  a.E = p.G1;  // G1 is consumed by the first factorisation
  a.X = p.Xw;
  a.R = p.R;
  a.R_out = R_out;
  a.ldr = ldr;
  a.refine = p.mixed;
  a.h = p.hdr;
  a.spin_limit = p.spin_limit;
  return a;
}

int dense_grid(const Plan& p) { return p.num_sms > 0 ? p.num_sms : 1; }

}  // namespace

int64_t wide_gram_part_doubles(int64_t m1, int n1, int64_t m2, int n2, int num_sms, int mixed) {
  int64_t most = 0;
  for (int pass = 1; pass <= 2; ++pass)
    for (int mask = 0; mask <= (mixed ? 6 : 0); mask += 2) {  // every choice of the tail blocks' engines
      WideBlock b[3];
      int gj = 0, fj = 0, tj = 0;
      int64_t pd = 0;
      wide_geometry(pass, m1, n1, m2, n2, num_sms, mask, b, &gj, &fj, &tj, &pd);
      if (pd > most) most = pd;
    }
  return most;
}

cudaError_t launch_wide_gram_pass(const Plan& p, int pass, cudaStream_t s) {
  WideArgs a{};
  const void* X[3] = {p.head, p.t[0].tail, p.t[1].tail};
  const int ld[3] = {p.n, p.n1, p.n2};
  // the tail blocks' Grams on the tensor cores (mixed path; the head block,
  // about one row per key group, stays on CUDA cores)
  int tc_mask = 0;
  if (p.mixed) {
    const int kq[3] = {p.n, pass == 1 ? p.n1 : p.n, p.n2};
    for (int i = 1; i < 3; ++i) {
      const void* G = pass == 1 ? X[i] : p.wq[i];
      const int64_t lg = pass == 1 ? ld[i] : kq[i];
      if (wide_tc_eligible(static_cast<const float*>(G), lg, kq[i])) tc_mask |= 1 << i;
    }
  }
  int tc_jobs = 0;
  int64_t part_doubles = 0;
  wide_geometry(pass, p.t[0].m, p.n1, p.t[1].m, p.n2, p.num_sms, tc_mask, a.b, &a.gram_jobs, &a.form_jobs, &tc_jobs,
                &part_doubles);
  const int es = p.mixed ? 4 : 8;
  for (int i = 0; i < 3; ++i) {
    a.b[i].X = X[i];
    a.b[i].ldx = ld[i];
    a.b[i].rows_dev = i == 0 ? &p.hdr->num_runs[0] : nullptr;
    a.b[i].Q = p.wq[i];
  }
  a.part = p.wpart;
  a.W = p.mixed ? static_cast<const void*>(p.Wf) : static_cast<const void*>(p.W);
  a.wld = p.n;
  a.G = pass == 1 ? p.G1 : p.G2;
  a.n = p.n;
  (void)es;
  // pass 2, mixed path: the tail blocks' formations on the tensor cores (W^T
  // and its lo parts prepared once), the rest on CUDA cores
  WideFormBlock fb[3];
  int form_tc = 0;
  if (pass == 2 && p.mixed && p.wt && p.n % 4 == 0) {
    for (int i = 0; i < 3; ++i) {
      WideBlock& B = a.b[i];
      fb[i] = WideFormBlock{};
      if (i == 0 || B.rows <= 0 || B.kout % 4 != 0 || !wide_tc_eligible(static_cast<const float*>(X[i]), ld[i], B.k))
        continue;
      const int ctiles = (B.kout + 127) / 128;
      const int nrt = static_cast<int>((B.rows + 127) / 128);
      int splits = (2 * p.num_sms + ctiles - 1) / ctiles;
      if (splits > nrt) splits = nrt;
      if (splits < 1) splits = 1;
      const int rps = (nrt + splits - 1) / splits;
      splits = (nrt + rps - 1) / rps;
      fb[i] = WideFormBlock{static_cast<const float*>(X[i]), ld[i], B.k, B.kout, B.w0, B.rows, B.rows_dev,
                            static_cast<float*>(p.wq[i]), ctiles, splits, rps, ctiles * splits};
      B.fjobs = 0;  // not for the CUDA-core formation
      form_tc += fb[i].njobs;
    }
    if (form_tc > 0) {
      int fj = 0;
      for (int i = 0; i < 3; ++i) {
        a.b[i].fjob0 = fj;
        fj += a.b[i].fjobs;
      }
      a.form_jobs = fj;
      cudaError_t err = launch_wide_form_prep(p.Wf, p.n, p.wt, p.wtlo, s);
      if (err != cudaSuccess) return err;
      err = launch_wide_form_tc(fb, p.wt, p.wtlo, p.n, &p.hdr->status, p.spin_limit, s);
      if (err != cudaSuccess) return err;
    }
  }
  if (pass == 2 && (a.form_jobs > 0 || form_tc > 0)) {
    if (a.form_jobs > 0) {
      if (p.mixed)
        pdl_launch(wide_form_kernel<float>, a.form_jobs, kWThreads, 0, s, a);
      else
        pdl_launch(wide_form_kernel<double>, a.form_jobs, kWThreads, 0, s, a);
      count_launches(1);
    }
    // the Grams of pass 2 read Q
    for (int i = 0; i < 3; ++i) {
      a.b[i].X = p.wq[i];
      a.b[i].ldx = a.b[i].kout;
    }
  }
  if (a.gram_jobs > 0) {
    if (p.mixed)
      pdl_launch(wide_gram_kernel<float>, a.gram_jobs, kWThreads, 0, s, a);
    else
      pdl_launch(wide_gram_kernel<double>, a.gram_jobs, kWThreads, 0, s, a);
    count_launches(1);
  }
  if (tc_jobs > 0) {
    WideTcBlock tb[3];
    for (int i = 0; i < 3; ++i) {
      const WideBlock& B = a.b[i];
      tb[i] = WideTcBlock{static_cast<const float*>(B.X), B.ldx, B.kout, B.rows, B.rows_dev, B.tc_tiles, B.tc_splits,
                          B.tc_split_rows, B.tc ? B.tc_njobs : 0, B.pbase};
    }
    const cudaError_t err = launch_wide_gram_tc(tb, p.wpart, &p.hdr->status, p.spin_limit, s);
    if (err != cudaSuccess) return err;
  }
  const int64_t ne = static_cast<int64_t>(p.n) * p.n;
  pdl_launch(wide_reduce_kernel, static_cast<int>((ne + kWThreads - 1) / kWThreads), kWThreads, 0, s, a);
  count_launches(1);
  return cudaGetLastError();
}

// Narrow mixed plans with n in (64, 128]: the Gram blocks with n output
// columns, more than the narrow tensor-core engines take, on the tile Gram
// (one 128 x 128 tile pair; partials [splits][128][128] in p.gpart[b],
// format 3 of the reduce): the head rows in pass 1 (X = the head rows, their
// count read on the device) and, after the tensor-core formation Q = X W into
// p.wq[b], the head rows and the A tails in pass 2.
static const float* narrow_tc_x(const Plan& p, int b, int64_t* ld, int* k) {
  *ld = b == 0 ? p.n : p.n1;
  *k = b == 0 ? p.n : p.n1;
  return static_cast<const float*>(b == 0 ? p.head : p.t[0].tail);
}

bool narrow_tc(const Plan& p, int pass, int b) {
  if (!(b == 0 || (b == 1 && pass == 2))) return false;
  if (!(p.mixed && !p.wide && p.gram_engine != 1 && p.n > 64 && p.n <= kWideTcTile && p.n % 4 == 0 &&
        p.n1 % 4 == 0 && p.t[0].m > 0 && p.wt && p.wq[b]))
    return false;
  // (the partial buffer must hold at least one 128 x 128 tile)
  if (p.gcap[b] < static_cast<int64_t>(kWideTcTile) * kWideTcTile) return false;
  int64_t ld = 0;
  int k = 0;
  const float* X = narrow_tc_x(p, b, &ld, &k);
  return wide_tc_eligible(X, ld, k);
}

int narrow_tc_splits(const Plan& p, int b, int64_t rows_min, int64_t* split_rows) {
  const int64_t rows = p.t[0].m;  // (head rows: at most m1, their count read on the device)
  const int64_t per = rows_min > 1024 ? rows_min : 1024;
  const int64_t cap = p.gcap[b] / (static_cast<int64_t>(kWideTcTile) * kWideTcTile);
  int64_t splits = (rows + per - 1) / per;
  if (splits > 2 * static_cast<int64_t>(p.num_sms)) splits = 2 * static_cast<int64_t>(p.num_sms);
  if (splits > cap) splits = cap;
  if (splits < 1) splits = 1;
  int64_t sr = (rows + splits - 1) / splits;
  sr = (sr + 127) / 128 * 128;  // whole row tiles of the formation
  *split_rows = sr;
  return static_cast<int>((rows + sr - 1) / sr);
}

void narrow_tc_blocks(const Plan& p, int pass, int b, int64_t rows_min, WideFormBlock* fb, WideTcBlock* tb) {
  const int n = p.n;
  const int64_t rows = p.t[0].m;
  const int64_t* rows_dev = b == 0 ? &p.hdr->num_runs[0] : nullptr;
  int64_t ld = 0;
  int k = 0;
  const float* X = narrow_tc_x(p, b, &ld, &k);
  int64_t sr = 0;
  const int splits = narrow_tc_splits(p, b, rows_min, &sr);
  *fb = WideFormBlock{};
  if (pass == 2) {  // formation: one CTA per split of sr / 128 row tiles (the Gram's splits)
    const int rps = static_cast<int>(sr / 128);
    *fb = WideFormBlock{X, ld, k, n, 0, rows, rows_dev, static_cast<float*>(p.wq[b]), 1, splits, rps, splits};
    fb->WT = p.wt;
    fb->WTlo = p.wtlo;
    fb->n = n;
    fb->status = &p.hdr->status;
    X = static_cast<const float*>(p.wq[b]);
    ld = n;
  }
  *tb = WideTcBlock{X, ld, n, rows, rows_dev, 1, splits, sr, splits, 0};
  tb->part = p.gpart[b];
  tb->status = &p.hdr->status;
}

cudaError_t launch_narrow_tc(const Plan& p, int pass, const bool use[3], int count[3], cudaStream_t s) {
  WideFormBlock fb[3] = {};
  WideTcBlock tb[3] = {};
  bool form = false;
  for (int b = 0; b < 2; ++b) {
    count[b] = 0;
    if (!use[b]) continue;
    narrow_tc_blocks(p, pass, b, 0, &fb[b], &tb[b]);
    // one launch for both blocks: partials of block 1 at their offset from block 0's buffer (one workspace)
    tb[b].pbase = p.gpart[b] - p.gpart[0];
    count[b] = tb[b].njobs;
    form = form || fb[b].njobs > 0;
  }
  cudaError_t err;
  if (form) {
    err = launch_wide_form_prep(p.Wf, p.n, p.wt, p.wtlo, s);
    if (err != cudaSuccess) return err;
    err = launch_wide_form_tc(fb, p.wt, p.wtlo, p.n, &p.hdr->status, p.spin_limit, s);
    if (err != cudaSuccess) return err;
  }
  return launch_wide_gram_tc(tb, p.gpart[0], &p.hdr->status, p.spin_limit, s);
}

static cudaError_t wide_first(const Plan& p, int from_r, cudaStream_t s) {
  DenseArgs a = dense_args(p, 0, nullptr, 0);
  if (from_r) {
    a.G = p.R;
    a.from_r = 1;
  } else if (p.shifted) {
    // 10 n u trace(G1), u the unit roundoff of the Gram products
    a.shift_rel = 10.0 * p.n * (p.mixed ? 5.9604644775390625e-8 : 1.1102230246251565e-16);
  }
  const size_t wsm = static_cast<size_t>(kWThreads / 32) * p.n * (p.mixed ? 4 : 8);
  cudaError_t err;
  if (p.mixed) {
    err = cudaFuncSetAttribute(wide_chol_first_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               static_cast<int>(wsm));
    if (err != cudaSuccess) return err;
    err = launch_cooperative(wide_chol_first_kernel<float>, dense_grid(p), kWThreads, wsm, s, a);
  } else {
    err = cudaFuncSetAttribute(wide_chol_first_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               static_cast<int>(wsm));
    if (err != cudaSuccess) return err;
    err = launch_cooperative(wide_chol_first_kernel<double>, dense_grid(p), kWThreads, wsm, s, a);
  }
  count_launches(1);
  return err;
}

cudaError_t launch_wide_chol_first(const Plan& p, cudaStream_t s) { return wide_first(p, 0, s); }

cudaError_t launch_wide_refactor(const Plan& p, cudaStream_t s) { return wide_first(p, 1, s); }

cudaError_t launch_wide_chol_second(const Plan& p, double* R_out, int64_t ldr, cudaStream_t s) {
  DenseArgs a = dense_args(p, 1, R_out, ldr);
  cudaError_t err = p.mixed ? launch_cooperative(wide_chol_second_kernel<float>, dense_grid(p), kWThreads, 0, s, a)
                            : launch_cooperative(wide_chol_second_kernel<double>, dense_grid(p), kWThreads, 0, s, a);
  count_launches(1);
  return err;
}

template <typename T, bool kWithV, int JW>
cudaError_t launch_jacobi_w(const Plan& p, JacArgs a, cudaStream_t s) {
  int nblk = (a.n + JW - 1) / JW;
  nblk += nblk & 1;
  a.nblk = nblk;
  // S (2 JW columns, stride n + 1), the row-split partial Grams, G and Q
  constexpr size_t W2 = 2 * JW, KS = 32 * JW / ((W2 / 4) * (W2 / 4));
  const size_t smem = sizeof(T) * (W2 * (static_cast<size_t>(a.n) + 1) + KS * W2 * W2 + 2 * W2 * (W2 + 1) + W2 * W2);
  if (nblk > kMaxJacobiBlocks) return cudaErrorInvalidValue;
  cudaError_t err = cudaFuncSetAttribute(wide_jacobi_kernel<T, kWithV, JW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  return launch_cooperative(wide_jacobi_kernel<T, kWithV, JW>, nblk / 2, 32 * JW, smem, s, a);
}

// sigma and V of R for any width: the block Jacobi with accumulated
// rotations (FP32 sweeps + FP64 Rayleigh quotients on the mixed path, FP64
// sweeps on the plain path).
cudaError_t launch_svd_v(const Plan& p, const double* R, int64_t ldr, double* sigma, double* V, int64_t ldv,
                         cudaStream_t s) {
  const int n = p.n;
  JacArgs a{};
  a.R = R;
  a.ldr = ldr;
  a.n = n;
  a.max_sweeps = p.max_sweeps;
  a.tol = p.mixed ? 1e-5 : 4.0 * n * 1.1102230246251565e-16;
  a.U = p.Uw;
  a.V = p.Vw;
  a.h = p.hdr;
  a.spin_limit = p.spin_limit;
  cudaError_t err;
  if (p.mixed) {
    err = launch_jacobi_w<float, true, 16>(p, a, s);
    if (err != cudaSuccess) return err;
    pdl_launch(wide_sigma_kernel<float, true>, n, kWThreads, 0, s, R, ldr, n, static_cast<const float*>(p.Uw),
               static_cast<const float*>(p.Vw), p.sigw, p.sigw + n, static_cast<const int32_t*>(&p.hdr->status));
    pdl_launch(wide_sort_v_kernel<float>, 1, kMaxWideWidth, 0, s, static_cast<const double*>(p.sigw),
               static_cast<const double*>(p.sigw + n), n, static_cast<const float*>(p.Vw), sigma, V, ldv,
               static_cast<const int32_t*>(&p.hdr->status));
  } else {
    err = launch_jacobi_w<double, true, 4>(p, a, s);
    if (err != cudaSuccess) return err;
    pdl_launch(wide_sigma_kernel<double, true>, n, kWThreads, 0, s, R, ldr, n, static_cast<const double*>(p.Uw),
               static_cast<const double*>(p.Vw), p.sigw, p.sigw + n, static_cast<const int32_t*>(&p.hdr->status));
    pdl_launch(wide_sort_v_kernel<double>, 1, kMaxWideWidth, 0, s, static_cast<const double*>(p.sigw),
               static_cast<const double*>(p.sigw + n), n, static_cast<const double*>(p.Vw), sigma, V, ldv,
               static_cast<const int32_t*>(&p.hdr->status));
  }
  count_launches(3);
  return cudaGetLastError();
}

cudaError_t launch_wide_jacobi(const Plan& p, const double* R, int64_t ldr, double* sigma, cudaStream_t s) {
  const int n = p.n;
  JacArgs a{};
  a.R = R;
  a.ldr = ldr;
  a.n = n;
  a.max_sweeps = p.max_sweeps;
  // FP32 sweeps stop at |u_p . u_q| <= 1e-5 ||u_p|| ||u_q||; the FP64
  // Rayleigh quotients then carry a relative error of order 1e-10 / gap
  a.tol = p.mixed ? 1e-5 : 4.0 * n * 1.1102230246251565e-16;
  a.U = p.Uw;
  a.V = p.Vw;
  a.h = p.hdr;
  a.spin_limit = p.spin_limit;
  cudaError_t err;
  if (p.mixed) {
    // FP32 sweeps: blocks of 16 columns (n / 32 CTAs of 16 warps; narrower
    // blocks double the rounds, whose barrier and staging costs dominate)
    err = launch_jacobi_w<float, true, 16>(p, a, s);
    if (err != cudaSuccess) return err;
    pdl_launch(wide_sigma_kernel<float, true>, n, kWThreads, 0, s, R, ldr, n, static_cast<const float*>(p.Uw),
                                                           static_cast<const float*>(p.Vw), p.sigw, p.sigw + n,
                                                           &p.hdr->status);
  } else {
    // FP64 sweeps are bound by the FP64 pipes: blocks of 4 columns spread
    // them over n / 8 CTAs
    err = launch_jacobi_w<double, false, 4>(p, a, s);
    if (err != cudaSuccess) return err;
    pdl_launch(wide_sigma_kernel<double, false>, n, kWThreads, 0, s, R, ldr, n, static_cast<const double*>(p.Uw),
                                                             static_cast<const double*>(p.Vw), p.sigw, p.sigw + n,
                                                             &p.hdr->status);
  }
  pdl_launch(wide_sort_kernel, 1, kMaxWideWidth, 0, s, p.sigw, p.sigw + n, n, sigma, &p.hdr->status);
  count_launches(3);
  return cudaGetLastError();
}

}  // namespace figaro
