// Gram products of the reduced matrix on CUDA cores (CholeskyQR2 passes).
//
// The reduced matrix M has three blocks stored separately (head rows, A's
// tail rows, B's tail rows), so M^T M is the sum of three smaller Grams:
//   pass 1:  G1 = Hd^T Hd + [TA^T TA, 0; 0, TB^T TB]
//   pass 2:  G2 = Q^T Q with Q = M W, W = R1^{-1} (upper triangular):
//            head rows   Hd W           (all n columns)
//            A tail rows TA W[0:n1, :]  (all n columns)
//            B tail rows TB W[n1:, n1:] (B's n2 columns only, since W is
//                                        upper triangular)
// Each block accumulates 4x4 register tiles of (X W)^T (X W) over 64-row
// tiles staged in shared memory.  On the mixed path the tiles are FP32 and
// are flushed into FP64 every 16 row tiles, so FP32 sums never run over more
// than 1,024 rows; the plain path accumulates in FP64 throughout.
// Partials go to [grid][slice] buffers and are reduced in a fixed order, so
// results are bitwise reproducible.
#include "common.cuh"
#include "internal.h"

namespace figaro {
namespace {

struct GramArgs {
  const void* X;          // rows x k (compute type), leading dimension ld
  int64_t ld;
  int k;
  int64_t rows;           // used when rows_dev == nullptr
  const int64_t* rows_dev;
  const void* W;          // optional n x n row-major (compute type)
  int wld;
  int wrow0, wcol0;       // the k x kout block of W used
  int kout;
  int kpad;               // kout rounded up to 4
  int tiles;              // (kpad/4)^2 register tiles
  int slices;             // thread groups splitting the rows of a tile
  int tile_rows;
  double* part;           // [grid][slices][kout][kout]
};

constexpr int kFlushTiles = 16;

template <typename T, int TPT>
__global__ void __launch_bounds__(kGramThreads) gram_kernel(GramArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Xs = reinterpret_cast<T*>(smem_raw);                          // tile_rows x k
  T* Ws = Xs + static_cast<int64_t>(a.tile_rows) * a.k;            // k x kpad (if W)
  T* Qs = a.W ? Ws + static_cast<int64_t>(a.k) * a.kpad : nullptr; // tile_rows x kpad
  const int RT = a.tile_rows;
  const int k = a.k, kp = a.kpad, T4 = kp / 4;
  const int64_t rows = a.rows_dev ? *a.rows_dev : a.rows;
  const T* X = static_cast<const T*>(a.X);
  const int tid = threadIdx.x;

  if (a.W) {
    const T* W = static_cast<const T*>(a.W);
    for (int e = tid; e < k * kp; e += blockDim.x) {
      int l = e / kp, c = e % kp;
      Ws[e] = c < a.kout ? W[static_cast<int64_t>(a.wrow0 + l) * a.wld + a.wcol0 + c] : T(0);
    }
  }
  const T* Q = a.W ? Qs : Xs;
  const int qld = a.W ? kp : k;

  // thread -> (slice, register tiles)
  int slice, tile0;
  if (TPT == 1) {
    slice = tid / a.tiles;
    tile0 = tid % a.tiles;
  } else {
    slice = 0;
    tile0 = tid;
  }
  const bool active = slice < a.slices;
  int ti[TPT], tj[TPT];
  bool tv[TPT];
#pragma unroll
  for (int q = 0; q < TPT; ++q) {
    int t = tile0 + q * kGramThreads;
    tv[q] = active && t < a.tiles;
    ti[q] = tv[q] ? t / T4 : 0;
    tj[q] = tv[q] ? t % T4 : 0;
  }
  T acc[TPT][4][4];
  double tot[TPT][4][4];
#pragma unroll
  for (int q = 0; q < TPT; ++q)
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        acc[q][i][j] = T(0);
        tot[q][i][j] = 0.0;
      }

  const int64_t ntiles = (rows + RT - 1) / RT;
  int since_flush = 0;
  for (int64_t rt = blockIdx.x; rt < ntiles; rt += gridDim.x) {
    __syncthreads();
    const int64_t r0 = rt * RT;
    // stage rows (zero beyond the end)
    for (int e = tid; e < RT * k; e += blockDim.x) {
      int r = e / k, c = e % k;
      int64_t gr = r0 + r;
      Xs[e] = gr < rows ? X[gr * a.ld + c] : T(0);
    }
    __syncthreads();
    if (a.W) {
      for (int e = tid; e < RT * kp; e += blockDim.x) {
        int r = e / kp, c = e % kp;
        T s = T(0);
        const T* xr = Xs + r * k;
        for (int l = 0; l < k; ++l) s += xr[l] * Ws[l * kp + c];
        Qs[e] = s;
      }
      __syncthreads();
    }
    if (active) {
      for (int r = slice; r < RT; r += a.slices) {
        const T* qr = Q + r * qld;
#pragma unroll
        for (int q = 0; q < TPT; ++q) {
          if (!tv[q]) continue;
          T u[4], w[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            int ci = ti[q] * 4 + i, cj = tj[q] * 4 + i;
            u[i] = (a.W || ci < k) ? qr[ci] : T(0);
            w[i] = (a.W || cj < k) ? qr[cj] : T(0);
          }
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[q][i][j] += u[i] * w[j];
        }
      }
    }
    if (++since_flush == kFlushTiles) {
      since_flush = 0;
#pragma unroll
      for (int q = 0; q < TPT; ++q)
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            tot[q][i][j] += static_cast<double>(acc[q][i][j]);
            acc[q][i][j] = T(0);
          }
    }
  }
  if (!active) return;
  double* out = a.part + (static_cast<int64_t>(blockIdx.x) * a.slices + slice) * a.kout * a.kout;
#pragma unroll
  for (int q = 0; q < TPT; ++q) {
    if (!tv[q]) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int ci = ti[q] * 4 + i, cj = tj[q] * 4 + j;
        if (ci < a.kout && cj < a.kout) out[ci * a.kout + cj] = tot[q][i][j] + static_cast<double>(acc[q][i][j]);
      }
  }
}

struct ReduceArgs {
  const double* part[3];
  int count[3];   // grid * slices partials per block
  int kout[3];
  int off[3];     // diagonal offset of the block inside G
  int n;
  double* G;
};

// G = sum of the three blocks' partials, in a fixed order (deterministic),
// symmetrised from the upper triangle.
__global__ void gram_reduce_kernel(ReduceArgs a) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.n * a.n) return;
  int i = e / a.n, j = e % a.n;
  int lo = i < j ? i : j, hi = i < j ? j : i;
  double s = 0.0;
  for (int b = 0; b < 3; ++b) {
    if (!a.part[b]) continue;
    int ii = lo - a.off[b], jj = hi - a.off[b];
    int ko = a.kout[b];
    if (ii < 0 || jj < 0 || ii >= ko || jj >= ko) continue;
    const double* p = a.part[b] + ii * ko + jj;
    const int64_t stride = static_cast<int64_t>(ko) * ko;
    double t = 0.0;
    for (int c = 0; c < a.count[b]; ++c) t += p[c * stride];
    s += t;
  }
  a.G[e] = s;
}

template <typename T>
cudaError_t launch_gram_block(const GramArgs& a0, int grid, cudaStream_t s) {
  GramArgs a = a0;
  size_t smem = static_cast<size_t>(a.tile_rows) * a.k * sizeof(T);
  if (a.W) smem += (static_cast<size_t>(a.k) * a.kpad + static_cast<size_t>(a.tile_rows) * a.kpad) * sizeof(T);
  int tpt = a.tiles <= kGramThreads ? 1 : (a.tiles <= 2 * kGramThreads ? 2 : 4);
  cudaError_t err;
  if (tpt == 1) {
    err = cudaFuncSetAttribute(gram_kernel<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    gram_kernel<T, 1><<<grid, kGramThreads, smem, s>>>(a);
  } else if (tpt == 2) {
    err = cudaFuncSetAttribute(gram_kernel<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    gram_kernel<T, 2><<<grid, kGramThreads, smem, s>>>(a);
  } else {
    err = cudaFuncSetAttribute(gram_kernel<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    gram_kernel<T, 4><<<grid, kGramThreads, smem, s>>>(a);
  }
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

// Geometry of one Gram block (shared with the workspace planner).
void gram_geometry(int kout, int* kpad, int* tiles, int* slices) {
  *kpad = (kout + 3) / 4 * 4;
  int T4 = *kpad / 4;
  *tiles = T4 * T4;
  *slices = *tiles <= kGramThreads ? kGramThreads / *tiles : 1;
}

int gram_tile_rows(int k, int kout, int with_w, int elem) {
  int kp = (kout + 3) / 4 * 4;
  for (int rt = kGramTileRows; rt >= 8; rt /= 2) {
    size_t smem = static_cast<size_t>(rt) * k * elem;
    if (with_w) smem += (static_cast<size_t>(k) * kp + static_cast<size_t>(rt) * kp) * elem;
    if (smem <= 200 * 1024) return rt;
  }
  return 8;
}

cudaError_t launch_gram_pass(const Plan& p, int pass, cudaStream_t s) {
  const int elem = p.mixed ? 4 : 8;
  // block 0 = head rows, 1 = A tails, 2 = B tails
  ReduceArgs r{};
  r.n = p.n;
  r.G = pass == 1 ? p.G1 : p.G2;
  for (int b = 0; b < 3; ++b) {
    GramArgs a{};
    int64_t rows;
    if (b == 0) {
      a.X = p.head;
      a.ld = p.n;
      a.k = p.n;
      a.rows_dev = &p.hdr->num_runs[0];
      rows = p.t[0].m;
    } else {
      const TableWork& T = p.t[b - 1];
      a.X = T.tail;
      a.ld = T.n;
      a.k = T.n;
      a.rows = T.m;
      rows = T.m;
    }
    if (rows == 0) continue;
    if (pass == 2) {
      a.W = p.mixed ? static_cast<const void*>(p.Wf) : static_cast<const void*>(p.W);
      a.wld = p.n;
      a.wrow0 = b == 2 ? p.n1 : 0;
      a.wcol0 = b == 2 ? p.n1 : 0;
      a.kout = b == 2 ? p.n2 : p.n;
    } else {
      a.kout = a.k;
    }
    gram_geometry(a.kout, &a.kpad, &a.tiles, &a.slices);
    a.tile_rows = gram_tile_rows(a.k, a.kout, a.W != nullptr, elem);
    a.part = p.gpart[b];
    int grid = p.ggrid[b];
    cudaError_t err = p.mixed ? launch_gram_block<float>(a, grid, s) : launch_gram_block<double>(a, grid, s);
    if (err != cudaSuccess) return err;
    r.part[b] = p.gpart[b];
    r.count[b] = grid * a.slices;
    r.kout[b] = a.kout;
    r.off[b] = b == 2 ? p.n1 : 0;
  }
  int ne = p.n * p.n;
  gram_reduce_kernel<<<(ne + 255) / 256, 256, 0, s>>>(r);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace figaro
