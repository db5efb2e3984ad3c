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
// A block streams 64-row tiles of X into shared memory (the next tile is
// prefetched into registers while the current one is used), forms Q = X W
// for the tile (W is upper triangular, so column c sums rows 0..c only) and
// accumulates the upper 4x4 register tiles of Q^T Q.  On the mixed path the
// register tiles are FP32 and are flushed into FP64 every 16 row tiles, so
// no FP32 sum runs over more than 1,024 rows; the plain path accumulates in
// FP64.  Thread groups (slices) that split the rows are summed inside the
// block in a fixed order, and the per-block partials are reduced in a fixed
// order as well: results are bitwise reproducible.
#include "common.cuh"
#include "internal.h"

namespace figaro {
namespace {

struct GramArgs {
  const void* X;          // rows x k (compute type), rows contiguous (leading dimension k)
  int k;
  int64_t rows;           // used when rows_dev == nullptr
  const int64_t* rows_dev;
  const void* W;          // optional n x n row-major (compute type)
  int wld;
  int w0;                 // the k x kout block W[w0:w0+k, w0:w0+kout] is used
  int kout;
  int kpad;               // kout rounded up to 4
  int ntiles;             // upper register tiles (T4 (T4+1) / 2)
  int slices;             // thread groups splitting the rows of a tile
  int tile_rows;
  double* part;           // [grid][kout][kout] (upper 4x4 tiles written)
};

constexpr int kFlushTiles = 16;

__device__ __forceinline__ void tile_of(int t, int T4, int& ti, int& tj) {
  // t -> (ti, tj), ti <= tj, row-wise over the upper triangle of a T4 x T4 grid
  ti = 0;
  int rowlen = T4;
  while (t >= rowlen) {
    t -= rowlen;
    ++ti;
    --rowlen;
  }
  tj = ti + t;
}

// 16-byte asynchronous global -> shared copy; bytes beyond src_bytes are zero-filled.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <typename T, int TPT>
__device__ __forceinline__ void gram_body(const GramArgs& a, int bid, int nb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int RT = a.tile_rows, k = a.k, kp = a.kpad, T4 = kp / 4;
  T* Xb[2] = {reinterpret_cast<T*>(smem_raw), reinterpret_cast<T*>(smem_raw) + RT * k};  // RT x k, two stages
  T* Ws = Xb[1] + RT * k;                                           // k x kp (if W)
  T* Qs = Ws + k * kp;                                              // RT x kp (if W)
  const int qld = a.W ? kp : k;
  const int64_t rows = a.rows_dev ? *a.rows_dev : a.rows;
  const char* X = static_cast<const char*>(a.X);
  const int tid = threadIdx.x;
  const int64_t total_bytes = rows * k * static_cast<int64_t>(sizeof(T));
  const int tile_bytes = RT * k * static_cast<int>(sizeof(T));  // a multiple of 16 (RT % 4 == 0)
  auto stage = [&](int64_t rt, T* dst) {
    const int64_t base = rt * tile_bytes;
    for (int c = tid * 16; c < tile_bytes; c += kGramThreads * 16) {
      int64_t left = total_bytes - (base + c);
      int nb = left >= 16 ? 16 : (left > 0 ? static_cast<int>(left) : 0);
      cp_async16(reinterpret_cast<char*>(dst) + c, nb > 0 ? X + base + c : X, nb);
    }
    cp_async_commit();
  };

  if (a.W) {
    const T* W = static_cast<const T*>(a.W);
    for (int e = tid; e < k * kp; e += blockDim.x) {
      int l = e / kp, c = e - l * kp;
      Ws[e] = (c < a.kout && l <= c) ? W[static_cast<int64_t>(a.w0 + l) * a.wld + a.w0 + c] : T(0);
    }
  }

  // thread -> slice and its upper register tiles
  const int per_slice = (a.ntiles + TPT - 1) / TPT;
  const int slice = tid / per_slice;
  const int lt = tid - slice * per_slice;
  const bool active = slice < a.slices;
  int ti[TPT], tj[TPT];
  bool tv[TPT];
#pragma unroll
  for (int q = 0; q < TPT; ++q) {
    int t = lt + q * per_slice;
    tv[q] = active && t < a.ntiles;
    ti[q] = tj[q] = 0;
    if (tv[q]) tile_of(t, T4, ti[q], tj[q]);
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

  const int64_t ntiles_rows = (rows + RT - 1) / RT;
  int64_t rt = bid;
  if (rt < ntiles_rows) stage(rt, Xb[0]);
  int since_flush = 0;
  for (int buf = 0; rt < ntiles_rows; rt += nb, buf ^= 1) {
    cp_async_wait_all();
    __syncthreads();  // tile rt landed; the other buffer is free
    if (rt + nb < ntiles_rows) stage(rt + nb, Xb[buf ^ 1]);  // overlaps the work below
    const T* Xs = Xb[buf];
    if (a.W) {
      for (int e = tid; e < RT * kp; e += blockDim.x) {
        int r = e / kp, c = e - r * kp;
        int lmax = c < k - 1 ? c : k - 1;
        T s = T(0);
        const T* xr = Xs + r * k;
        for (int l = 0; l <= lmax; ++l) s += xr[l] * Ws[l * kp + c];
        Qs[e] = s;
      }
      __syncthreads();
    }
    if (active) {
      for (int r = slice; r < RT; r += a.slices) {
        const T* qr = (a.W ? static_cast<const T*>(Qs) : Xs) + r * qld;
#pragma unroll
        for (int q = 0; q < TPT; ++q) {
          if (!tv[q]) continue;
          T u[4], w[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            int ci = ti[q] * 4 + i, cj = tj[q] * 4 + i;
            u[i] = ci < qld ? qr[ci] : T(0);
            w[i] = cj < qld ? qr[cj] : T(0);
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
#pragma unroll
  for (int q = 0; q < TPT; ++q)
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) tot[q][i][j] += static_cast<double>(acc[q][i][j]);

  // slices summed in a fixed order in shared memory, then one partial per block
  cp_async_wait_all();
  __syncthreads();
  double* red = reinterpret_cast<double*>(smem_raw);  // kpad x kpad
  for (int e = tid; e < kp * kp; e += blockDim.x) red[e] = 0.0;
  for (int s = 0; s < a.slices; ++s) {
    __syncthreads();
    if (active && slice == s) {
#pragma unroll
      for (int q = 0; q < TPT; ++q) {
        if (!tv[q]) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) red[(ti[q] * 4 + i) * kp + tj[q] * 4 + j] += tot[q][i][j];
      }
    }
  }
  __syncthreads();
  double* out = a.part + static_cast<int64_t>(bid) * a.kout * a.kout;
  for (int e = tid; e < a.kout * a.kout; e += blockDim.x) {
    int i = e / a.kout, j = e - i * a.kout;
    out[e] = red[i * kp + j];
  }
}

template <typename T, int TPT>
__global__ void __launch_bounds__(kGramThreads) gram_kernel(GramArgs a) {
  pdl_enter();
  gram_body<T, TPT>(a, blockIdx.x, gridDim.x);
}

struct ReduceArgs {
  const double* part[3];
  int count[3];   // partials (blocks) per Gram block
  int kout[3];
  int off[3];     // diagonal offset of the block inside G
  int sym[3];     // partial format: 0 FP64 upper triangle; 1 FP64 P with G = (P + P^T) / 2 (general
                  // tensor-core engine); 2 float-float pairs, upper triangle (packed tensor-core engine);
                  // 3 FP64 upper triangle of 128 x 128 tiles (the tile Gram, one tile pair: kout <= 128)
  int n;
  double* G;
};


// G = sum of the three blocks' partials in a fixed order (deterministic).
// Two layouts: with many partials (kPerWarp false) a block owns 32
// consecutive outputs (one per lane) and its warps interleave over the
// partials, warp 0 adding the warps' sums; with few (batched calls, a few
// dozen per block) every warp owns 32 outputs and sums all their partials
// itself, so that a block covers 16 times as many outputs.  Each thread
// issues the loads of up to five partials of every block before its first
// addition (the loads are latency-bound).  Partials of the packed
// tensor-core engine are float-float pairs and are summed in float-float
// (FP64 arithmetic is slow on this GPU); the others are FP64.
template <bool kPerWarp>
__device__ __forceinline__ void gram_reduce_body(const ReduceArgs& a, int bid) {
  __shared__ double sd[kPerWarp ? 1 : kReduceWarps][33];
  __shared__ float2 sf[kPerWarp ? 1 : kReduceWarps][33];
  constexpr int kPer = 5;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int e = (kPerWarp ? bid * kReduceWarps + warp : bid) * 32 + lane;
  const int cfirst = kPerWarp ? 0 : warp, cstep = kPerWarp ? 1 : kReduceWarps;
  const bool ok = e < a.n * a.n;
  const int i = ok ? e / a.n : 0, j = ok ? e - (e / a.n) * a.n : 0;
  const int lo = i < j ? i : j, hi = i < j ? j : i;
  const unsigned long long* p0[3];
  const unsigned long long* p1[3];
  int64_t stride[3];
  int cnt[3];
  int maxc = 0;
  bool any64 = false;
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const int ko = a.kout[b];
    const int ii = lo - a.off[b], jj = hi - a.off[b];
    const bool in = a.part[b] && ok && ii >= 0 && jj >= 0 && ii < ko && jj < ko;
    cnt[b] = in ? a.count[b] : 0;
    const int pitch = a.sym[b] == 3 ? kWideTcTile : ko;
    stride[b] = static_cast<int64_t>(pitch) * pitch;
    const unsigned long long* base = reinterpret_cast<const unsigned long long*>(a.part[b]);
    p0[b] = in ? base + ii * pitch + jj : nullptr;
    p1[b] = in ? base + jj * pitch + ii : nullptr;  // the transposed entry (symmetrised partials)
    maxc = a.count[b] > maxc ? a.count[b] : maxc;
    any64 = any64 || (a.part[b] && a.sym[b] != 2);
  }
  double t[4] = {0.0, 0.0, 0.0, 0.0};
  float fh = 0.f, fl = 0.f;
  for (int c0 = 0; c0 < maxc; c0 += kPer * cstep) {
    unsigned long long v[3][kPer], w[3][kPer];
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int k = 0; k < kPer; ++k) {
        const int c = c0 + cfirst + k * cstep;
        const bool live = c < cnt[b];
        v[b][k] = live ? p0[b][c * stride[b]] : 0ull;
        w[b][k] = live && a.sym[b] == 1 ? p1[b][c * stride[b]] : 0ull;
      }
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int k = 0; k < kPer; ++k) {
        if (a.sym[b] == 2) {
          const float2 q = make_float2(__uint_as_float(static_cast<uint32_t>(v[b][k])),
                                       __uint_as_float(static_cast<uint32_t>(v[b][k] >> 32)));
          float s_, e_;
          two_sum(fh, q.x, s_, e_);
          fh = s_;
          fl = __fadd_rn(fl, __fadd_rn(e_, q.y));
        } else if (c0 + cfirst + k * cstep < cnt[b]) {
          const double d = __longlong_as_double(static_cast<long long>(v[b][k]));
          t[k & 3] += a.sym[b] == 1 ? 0.5 * (d + __longlong_as_double(static_cast<long long>(w[b][k]))) : d;
        }
      }
  }
  if (kPerWarp) {
    if (ok) a.G[e] = static_cast<double>(fh) + static_cast<double>(fl) + (any64 ? (t[0] + t[1]) + (t[2] + t[3]) : 0.0);
    return;
  }
  sd[warp][lane] = any64 ? (t[0] + t[1]) + (t[2] + t[3]) : 0.0;
  sf[warp][lane] = make_float2(fh, fl);
  __syncthreads();
  if (warp == 0 && ok) {
    float gh = 0.f, gl = 0.f;
#pragma unroll
    for (int w = 0; w < kReduceWarps; ++w) {
      const float2 q = sf[w][lane];
      float s_, e_;
      two_sum(gh, q.x, s_, e_);
      gh = s_;
      gl = __fadd_rn(gl, __fadd_rn(e_, q.y));
    }
    double g = static_cast<double>(gh) + static_cast<double>(gl);
    if (any64) {
      double u[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int w = 0; w < kReduceWarps; ++w) u[w & 3] += sd[w][lane];
      g += (u[0] + u[1]) + (u[2] + u[3]);
    }
    a.G[e] = g;
  }
}

__global__ void __launch_bounds__(32 * kReduceWarps) gram_reduce_kernel(ReduceArgs a) {
  pdl_enter();
  gram_reduce_body<false>(a, blockIdx.x);
}

// Geometry of one Gram block: kout padded to 4, the upper 4 x 4 register
// tiles, thread groups (slices) splitting a row tile, tiles per thread.
__host__ __device__ inline void gram_geom(int kout, int* kpad, int* ntiles, int* slices, int* tpt) {
  *kpad = (kout + 3) / 4 * 4;
  const int T4 = *kpad / 4;
  *ntiles = T4 * (T4 + 1) / 2;
  int t = 1;
  while ((*ntiles + t - 1) / t > kGramThreads) t <<= 1;
  *tpt = t;
  const int per_slice = (*ntiles + t - 1) / t;
  *slices = kGramThreads / per_slice;
}

__host__ __device__ inline int gram_rows_per_tile(int k, int kout, int with_w, int elem) {
  const int kp = (kout + 3) / 4 * 4;
  for (int rt = kGramTileRows; rt >= 4; rt /= 2) {
    size_t smem = 2 * static_cast<size_t>(rt) * k * elem;
    if (with_w) smem += (static_cast<size_t>(k) * kp + static_cast<size_t>(rt) * kp) * elem;
    if (smem <= 200 * 1024) return rt;
  }
  return 4;
}

__host__ __device__ inline size_t gram_smem_bytes(const GramArgs& a, int elem) {
  size_t smem = 2 * static_cast<size_t>(a.tile_rows) * a.k * elem;
  if (a.W) smem += (static_cast<size_t>(a.k) * a.kpad + static_cast<size_t>(a.tile_rows) * a.kpad) * elem;
  const size_t red = sizeof(double) * a.kpad * a.kpad;
  return smem < red ? red : smem;
}

// The CUDA-core arguments of Gram block b (0 head rows, 1 A tails, 2 B tails)
// of a pass; *rows_host = the block's row bound (0: the block is empty).
__host__ __device__ inline GramArgs gram_args_of(const Plan& p, int pass, int b, int64_t* rows_host, int* tpt) {
  GramArgs a{};
  if (b == 0) {
    a.X = p.head;
    a.k = p.n;
    a.rows_dev = &p.hdr->num_runs[0];
    *rows_host = p.t[0].m;
  } else {
    const TableWork& T = p.t[b - 1];
    a.X = T.tail;
    a.k = T.n;
    a.rows = T.m;
    *rows_host = T.m;
  }
  if (pass == 2) {
    a.W = p.mixed ? static_cast<const void*>(p.Wf) : static_cast<const void*>(p.W);
    a.wld = p.n;
    a.w0 = b == 2 ? p.n1 : 0;
    a.kout = b == 2 ? p.n2 : p.n;
  } else {
    a.kout = a.k;
  }
  gram_geom(a.kout, &a.kpad, &a.ntiles, &a.slices, tpt);
  a.tile_rows = gram_rows_per_tile(a.k, a.kout, a.W != nullptr, p.mixed ? 4 : 8);
  a.part = p.gpart[b];
  return a;
}

__host__ __device__ inline ReduceArgs reduce_args_of(const Plan& p, int pass) {
  ReduceArgs r{};
  r.n = p.n;
  r.G = pass == 1 ? p.G1 : p.G2;
  for (int b = 0; b < 3; ++b) {
    int64_t rows = 0;
    int tpt = 0;
    const GramArgs a = gram_args_of(p, pass, b, &rows, &tpt);
    if (rows == 0) continue;
    r.part[b] = p.gpart[b];
    r.count[b] = p.gcount[pass - 1][b] > 0 ? p.gcount[pass - 1][b] : p.ggrid[b];
    r.kout[b] = a.kout;
    r.off[b] = b == 2 ? p.n1 : 0;
    r.sym[b] = p.gsym[pass - 1][b];
  }
  return r;
}

// ---- batched forms (CUDA-core Gram): Gram jobs are (instance, block) with
// aux = block and p.ggrid[block] CTAs; reduce jobs are instances with
// aux = 1 and ceil(n^2 / 512) CTAs (a warp per 32 outputs) when every block
// has few partials, else aux = 0 and ceil(n^2 / 32) CTAs
// (the arguments of each CTA's job are precomputed on the host when `args`
// is set: computing them from the plan is a chain of dependent loads by one
// thread, which dominated launches of thousands of small CTAs)
template <typename A>
__device__ __forceinline__ void copy_args(A* dst, const A* src) {
  static_assert(sizeof(A) % 4 == 0, "word copy");
  const uint32_t* s_ = reinterpret_cast<const uint32_t*>(src);
  uint32_t* d_ = reinterpret_cast<uint32_t*>(dst);
  for (int w = threadIdx.x; w < static_cast<int>(sizeof(A) / 4); w += blockDim.x) d_[w] = s_[w];
}

template <typename T, int TPT>
__global__ void __launch_bounds__(kGramThreads) gram_batched(BatchDev bd, BatchJobs J, int pass, const GramArgs* args) {
  pdl_enter();
  __shared__ GramArgs s_a;
  const int j = batch_job(J, blockIdx.x);
  if (args) {
    copy_args(&s_a, args + static_cast<int64_t>(J.inst[j]) * 3 + J.aux[j]);
  } else if (threadIdx.x == 0) {
    int64_t rows = 0;
    int tpt = 0;
    s_a = gram_args_of(bd.plans[J.inst[j]], pass, J.aux[j], &rows, &tpt);
  }
  __syncthreads();
  gram_body<T, TPT>(s_a, blockIdx.x - J.first[j], J.first[j + 1] - J.first[j]);
}

__global__ void __launch_bounds__(32 * kReduceWarps) gram_reduce_batched(BatchDev bd, BatchJobs J, int pass,
                                                                        const ReduceArgs* args) {
  pdl_enter();
  __shared__ ReduceArgs s_r;
  const int j = batch_job(J, blockIdx.x);
  if (args) copy_args(&s_r, args + J.inst[j]);
  else if (threadIdx.x == 0) s_r = reduce_args_of(bd.plans[J.inst[j]], pass);
  __syncthreads();
  if (J.aux[j]) gram_reduce_body<true>(s_r, blockIdx.x - J.first[j]);  // few partials: a warp per 32 outputs
  else gram_reduce_body<false>(s_r, blockIdx.x - J.first[j]);
}

template <typename T>
cudaError_t launch_batch_gram_t(const BatchDev& b, int pass, const BatchJobs* by_tpt, const size_t* smem,
                                const BatchJobs& reduce, const void* gargs, const void* rargs, cudaStream_t s) {
  for (int q = 0; q < 4; ++q) {
    if (by_tpt[q].njobs == 0) continue;
    auto kern = q == 0 ? gram_batched<T, 1> : (q == 1 ? gram_batched<T, 2> : (q == 2 ? gram_batched<T, 4> : gram_batched<T, 8>));
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem[q]));
    if (err != cudaSuccess) return err;
    pdl_launch(kern, by_tpt[q].ctas, kGramThreads, smem[q], s, b, by_tpt[q], pass,
               static_cast<const GramArgs*>(gargs));
    count_launches(1);
  }
  if (reduce.njobs > 0) {
    pdl_launch(gram_reduce_batched, reduce.ctas, 32 * kReduceWarps, 0, s, b, reduce, pass,
               static_cast<const ReduceArgs*>(rargs));
    count_launches(1);
  }
  return cudaGetLastError();
}

template <typename T, int TPT>
cudaError_t launch_tpt(const GramArgs& a, int grid, size_t smem, cudaStream_t s) {
  cudaError_t err =
      cudaFuncSetAttribute(gram_kernel<T, TPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  pdl_launch(gram_kernel<T, TPT>, grid, kGramThreads, smem, s, a);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gram_block(const GramArgs& a, int tpt, int grid, cudaStream_t s) {
  const size_t smem = gram_smem_bytes(a, sizeof(T));
  switch (tpt) {
    case 1: return launch_tpt<T, 1>(a, grid, smem, s);
    case 2: return launch_tpt<T, 2>(a, grid, smem, s);
    case 4: return launch_tpt<T, 4>(a, grid, smem, s);
    default: return launch_tpt<T, 8>(a, grid, smem, s);
  }
}

}  // namespace

// Geometry of one Gram block (shared with the workspace planner).
void gram_geometry(int kout, int* kpad, int* ntiles, int* slices, int* tpt) { gram_geom(kout, kpad, ntiles, slices, tpt); }

int gram_tile_rows(int k, int kout, int with_w, int elem) { return gram_rows_per_tile(k, kout, with_w, elem); }

// Batched Gram jobs of one instance: for each block with rows, its
// tiles-per-thread variant (0..3 for 1, 2, 4, 8), CTAs and shared memory.
void gram_batch_block(const Plan& p, int pass, int b, int* variant, int* ctas, size_t* smem) {
  int64_t rows = 0;
  int tpt = 1;
  const GramArgs a = gram_args_of(p, pass, b, &rows, &tpt);
  *ctas = rows > 0 ? p.ggrid[b] : 0;
  *variant = tpt <= 1 ? 0 : (tpt == 2 ? 1 : (tpt == 4 ? 2 : 3));
  *smem = gram_smem_bytes(a, p.mixed ? 4 : 8);
}

cudaError_t launch_batch_gram(const BatchDev& b, int pass, const BatchJobs by_tpt[4], const size_t smem[4],
                              const BatchJobs& reduce, int mixed, const void* gargs, const void* rargs,
                              cudaStream_t s) {
  return mixed ? launch_batch_gram_t<float>(b, pass, by_tpt, smem, reduce, gargs, rargs, s)
               : launch_batch_gram_t<double>(b, pass, by_tpt, smem, reduce, gargs, rargs, s);
}

size_t batch_gram_args_bytes() { return sizeof(GramArgs); }
size_t batch_reduce_args_bytes() { return sizeof(ReduceArgs); }

namespace {
// One thread per (instance, block) and per instance for the reduce: each
// derives its job's arguments from the plan once, in parallel.
__global__ void batch_args_kernel(BatchDev bd, int pass, GramArgs* ga, ReduceArgs* ra) {
  pdl_enter();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 4 * bd.count) return;
  const int i = e >> 2, k = e & 3;
  if (k < 3) {
    int64_t rows = 0;
    int tpt = 0;
    ga[static_cast<int64_t>(i) * 3 + k] = gram_args_of(bd.plans[i], pass, k, &rows, &tpt);
  } else {
    ra[i] = reduce_args_of(bd.plans[i], pass);
  }
}
}  // namespace

cudaError_t launch_batch_args(const BatchDev& b, int pass, void* gargs, void* rargs, cudaStream_t s) {
  if (b.count == 0) return cudaSuccess;
  pdl_launch(batch_args_kernel, (4 * b.count + 255) / 256, 256, 0, s, b, pass, static_cast<GramArgs*>(gargs),
             static_cast<ReduceArgs*>(rargs));
  count_launches(1);
  return cudaGetLastError();
}

bool gram_tc_supported(int k, int kout);
bool gram_tc_packs(int k, int kout, bool pass2);
// X1, k1, rows1: pass 2, a second block with the same W block and Gram
// (its rows follow the first block's in one launch; k1 <= k)
cudaError_t launch_gram_tc_block(const void* X, int k, int64_t rows, const int64_t* rows_dev, const float* W, int wld,
                                 int kout, double* part, int grid_max, int num_sms, int* grid_used, int32_t* status,
                                 int64_t spin_limit, int withhold, cudaStream_t s, const void* X1 = nullptr, int k1 = 0,
                                 int64_t rows1 = 0);

cudaError_t launch_gram_pass(const Plan& p, int pass, cudaStream_t s) {
  if (p.wide) return launch_wide_gram_pass(p, pass, s);
  const int elem = p.mixed ? 4 : 8;
  // block 0 = head rows, 1 = A tails, 2 = B tails
  // n in (64, 128]: the blocks with n output columns on the tile Gram (one launch for both)
  bool ntc[3] = {false, false, false};
  int ncount[3] = {0, 0, 0};
  for (int b = 0; b < 2; ++b) ntc[b] = narrow_tc(p, pass, b);
  if (ntc[0] || ntc[1]) {
    const cudaError_t err = launch_narrow_tc(p, pass, ntc, ncount, s);
    if (err != cudaSuccess) return err;
  }
  ReduceArgs r{};
  r.n = p.n;
  r.G = pass == 1 ? p.G1 : p.G2;
  // pass 2, n <= 32 on the packed engine: the head rows' Q = H W and the A
  // tails' Q = T W[0:n1, :] have the same width and W block (the tails' K
  // columns past n1 read as zeros), so both run in one launch whose partials
  // hold their sum (the head block's fixed costs were most of its launch)
  const bool pair01 = pass == 2 && p.mixed && p.gram_engine != 1 && !ntc[0] && !ntc[1] && p.t[0].m > 0 &&
                      gram_tc_supported(p.n, p.n) && gram_tc_supported(p.n1, p.n) && gram_tc_packs(p.n, p.n, true) &&
                      gram_tc_packs(p.n1, p.n, true) && p.n1 <= p.n;
  for (int b = 0; b < 3; ++b) {
    if (pair01 && b == 1) continue;  // (launched with the head rows)
    GramArgs a{};
    int64_t rows;
    if (b == 0) {
      a.X = p.head;
      a.k = p.n;
      a.rows_dev = &p.hdr->num_runs[0];
      rows = p.t[0].m;
    } else {
      const TableWork& T = p.t[b - 1];
      a.X = T.tail;
      a.k = T.n;
      a.rows = T.m;
      rows = T.m;
    }
    if (rows == 0) continue;
    if (pass == 2) {
      a.W = p.mixed ? static_cast<const void*>(p.Wf) : static_cast<const void*>(p.W);
      a.wld = p.n;
      a.w0 = b == 2 ? p.n1 : 0;
      a.kout = b == 2 ? p.n2 : p.n;
    } else {
      a.kout = a.k;
    }
    int tpt;
    gram_geometry(a.kout, &a.kpad, &a.ntiles, &a.slices, &tpt);
    a.tile_rows = gram_tile_rows(a.k, a.kout, a.W != nullptr, elem);
    a.part = p.gpart[b];
    int grid = p.ggrid[b];
    if (pass == 1 && b >= 1 && p.ht_gram[b - 1] > 0) {  // partials written by the head/tail stream
      r.part[b] = p.gpart[b];
      r.count[b] = p.ht_gram[b - 1];
      r.kout[b] = a.kout;
      r.off[b] = b == 2 ? p.n1 : 0;
      r.sym[b] = 2;
      continue;
    }
    if (ntc[b]) {  // launched above
      r.part[b] = p.gpart[b];
      r.count[b] = ncount[b];
      r.kout[b] = a.kout;
      r.off[b] = 0;
      r.sym[b] = 3;
      continue;
    }
    const bool tc = p.mixed && p.gram_engine != 1 && gram_tc_supported(a.k, a.kout);
    cudaError_t err;
    if (tc) {
      const float* Wb = pass == 2 ? p.Wf + static_cast<int64_t>(a.w0) * p.n + a.w0 : nullptr;
      if (pair01 && b == 0)
        err = launch_gram_tc_block(a.X, a.k, rows, a.rows_dev, Wb, p.n, a.kout, a.part, p.ggrid[b], p.num_sms, &grid,
                                   &p.hdr->status, p.spin_limit, p.withhold, s, p.t[0].tail, p.n1, p.t[0].m);
      else
        err = launch_gram_tc_block(a.X, a.k, rows, a.rows_dev, Wb, p.n, a.kout, a.part, p.ggrid[b], p.num_sms, &grid,
                                   &p.hdr->status, p.spin_limit, p.withhold, s);
    } else {
      err = p.mixed ? launch_gram_block<float>(a, tpt, grid, s) : launch_gram_block<double>(a, tpt, grid, s);
    }
    if (err != cudaSuccess) return err;
    r.part[b] = p.gpart[b];
    r.count[b] = grid;
    r.kout[b] = a.kout;
    r.off[b] = b == 2 ? p.n1 : 0;
    r.sym[b] = tc ? (gram_tc_packs(a.k, a.kout, pass == 2) ? 2 : 1) : 0;
  }
  const int ne = p.n * p.n;
  pdl_launch(gram_reduce_kernel, (ne + 31) / 32, 32 * kReduceWarps, 0, s, r);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace figaro
