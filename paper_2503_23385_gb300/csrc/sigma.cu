// Singular values of an upper-triangular R without rotating R's columns
// (Section 3: when only the singular values are wanted, the square-root-free
// differential qd method, dqds, is the usual choice).  Two stages, one CTA
// per matrix (n <= 128, R staged in shared memory):
//
//  1. Golub-Kahan bidiagonalisation B = U^T R V by Householder reflections
//     from the left (zeroing column k below the diagonal) and the right
//     (zeroing row k beyond the superdiagonal), alternately, k = 0 .. n-1.
//     U and V are not formed.  Orthogonal transformations keep the singular
//     values; the backward error is of order u ||R|| (u the unit roundoff).
//  2. dqds (Rutishauser's quotient-difference recurrence in the differential
//     form of Fernando and Parlett, 1994) on the squares q_i = b_ii^2 and
//     e_i = b_i,i+1^2: each transform with shift tau maps the qd array of
//     B^T B to that of B^T B - tau I with only positive terms when tau lies
//     below the smallest eigenvalue, which keeps every value to high relative
//     accuracy.  The shifts accumulate in S; when the last e falls below
//     u^2 (S + q_last) / 9 the last eigenvalue S + q_last has converged and
//     the array shrinks by one (an interior e below u^2 S / 9 splits it).
//
// The shift: warp 0 runs the transform for 32 shifts at once, one per lane,
// tau_l = est (1 - g_l) with est an upper bound of the smallest eigenvalue
// (the smaller of the last transform's smallest d and the smaller eigenvalue
// of the trailing 2 x 2 of B B^T, by interlacing) and g_l a geometric ladder
// from u to 1/2 with g_31 = 1 (tau = 0, which always succeeds), and keeps
// the largest tau whose transform stayed positive: a rejected shift costs no
// extra pass, as it would in a serial search.
//
// Precision.  Dependent FP64 operations are slow on this GPU (each step of
// the dqds recurrence is a chain of an add, a divide and a multiply-add), so
// the recurrence never runs in FP64: the accurate form (the FP64 path and
// figaro_triangular_singular_values) bidiagonalises in FP64 and runs dqds in
// float-float (pairs of FP32 values, about 46 significant bits: Dekker's
// products and Knuth's sums), the fast form (the mixed path) runs both
// stages in FP32 (normwise error of order 2^-24 ||R||).
#include <cfloat>

#include "internal.h"

namespace figaro {
namespace {

constexpr int kSigThreads = 256;
constexpr int kSigWarps = kSigThreads / 32;
constexpr int kCand = 33;  // entries between i and i + 1 of a lane's candidate arrays (bank spread)

__host__ __device__ constexpr int sig_lda(int n) { return n | 1; }  // odd stride: column walks are conflict-free
__host__ __device__ constexpr size_t sig_al8(size_t b) { return (b + 7) & ~size_t(7); }
// Bytes of the first region: the matrix in T, later the lanes' candidate
// arrays (2 x kCand x n values of NT), and at least 8 doubles (a reduction).
template <typename T, typename NT>
__host__ __device__ constexpr size_t sig_region_bytes(int n) {
  return sig_al8(sizeof(T) * n * sig_lda(n) > sizeof(NT) * 2 * kCand * n ? sizeof(T) * n * sig_lda(n)
                                                                          : sizeof(NT) * 2 * kCand * n);
}

// ---------------------------------------------------------------- numbers --

// Float-float value h + l with |l| <= ulp(h) / 2.
struct FF {
  float h, l;
};

__device__ __forceinline__ FF ff_fast(float s, float e) {  // |s| >= |e|
  const float h = __fadd_rn(s, e);
  return {h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  float s, e, t, f;
  two_sum(a.h, b.h, s, e);
  two_sum(a.l, b.l, t, f);
  FF r = ff_fast(s, __fadd_rn(e, t));
  return ff_fast(r.h, __fadd_rn(r.l, f));
}
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
  return ff_fast(p, e);
}
__device__ __forceinline__ FF ff_div(FF a, FF b) {
  const float r = __fdividef(1.0f, b.h);  // ~1 ulp: the remainder step corrects q1
  const float q1 = __fmul_rn(a.h, r);
  const float p = __fmul_rn(q1, b.h), pe = __fmaf_rn(q1, b.h, -p);
  float s, e;
  two_sum(a.h, -p, s, e);  // s + e = a.h - p exactly
  e = __fmaf_rn(-q1, b.l, __fadd_rn(__fsub_rn(e, pe), a.l));
  return ff_fast(q1, __fmul_rn(__fadd_rn(s, e), r));
}
__device__ __forceinline__ FF ff_sqrt(FF a) {
  if (!(a.h > 0.0f)) return {0.0f, 0.0f};
  const float s = sqrtf(a.h);
  const float p = __fmul_rn(s, s), pe = __fmaf_rn(s, s, -p);
  float d, e;
  two_sum(a.h, -p, d, e);
  const float rem = __fadd_rn(d, __fadd_rn(__fsub_rn(e, pe), a.l));
  return ff_fast(s, __fdividef(rem, 2.0f * s));
}

// The arithmetic of the dqds stage.
struct FFNum {
  using T = FF;
  static constexpr int kBits = 46;  // roundoff of the float-float operations above, about 2^-46
  __device__ static T from(double x) {
    const float h = static_cast<float>(x);
    return {h, static_cast<float>(x - static_cast<double>(h))};
  }
  __device__ static double to_double(T a) { return static_cast<double>(a.h) + static_cast<double>(a.l); }
  __device__ static T add(T a, T b) { return ff_add(a, b); }
  __device__ static T sub(T a, T b) { return ff_add(a, {-b.h, -b.l}); }
  __device__ static T mul(T a, T b) { return ff_mul(a, b); }
  __device__ static T div(T a, T b) { return ff_div(a, b); }
  __device__ static T sqrt_(T a) { return ff_sqrt(a); }
  __device__ static T scale(T a, float p2) { return {a.h * p2, a.l * p2}; }  // exact for a power of two
  __device__ static bool pos(T a) { return a.h > 0.0f; }
  __device__ static bool nonneg(T a) { return a.h >= 0.0f; }
  __device__ static bool less(T a, T b) { return a.h < b.h || (a.h == b.h && a.l < b.l); }
  __device__ static bool leq(T a, T b) { return !less(b, a); }
  __device__ static T shfl(T a, int src) {
    return {__shfl_sync(0xffffffffu, a.h, src), __shfl_sync(0xffffffffu, a.l, src)};
  }
};

struct F32Num {
  using T = float;
  static constexpr int kBits = 23;
  __device__ static T from(double x) { return static_cast<float>(x); }
  __device__ static double to_double(T a) { return static_cast<double>(a); }
  __device__ static T add(T a, T b) { return a + b; }
  __device__ static T sub(T a, T b) { return a - b; }
  __device__ static T mul(T a, T b) { return a * b; }
  __device__ static T div(T a, T b) { return __fdividef(a, b); }  // ~2 ulp; |b| stays far below 2^126
  __device__ static T sqrt_(T a) { return sqrtf(fmaxf(a, 0.0f)); }
  __device__ static T scale(T a, float p2) { return a * p2; }
  __device__ static bool pos(T a) { return a > 0.0f; }
  __device__ static bool nonneg(T a) { return a >= 0.0f; }
  __device__ static bool less(T a, T b) { return a < b; }
  __device__ static bool leq(T a, T b) { return a <= b; }
  __device__ static T shfl(T a, int src) { return __shfl_sync(0xffffffffu, a, src); }
};

// ------------------------------------------------------ bidiagonalisation --

// Sum over the block; red holds kSigWarps values.  One barrier: callers
// alternate two red buffers so that a buffer is rewritten only after a
// later barrier.
template <typename T>
__device__ __forceinline__ T sig_block_sum(T v, T* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  T s = T(0);
#pragma unroll
  for (int w = 0; w < kSigWarps; ++w) s += red[w];
  return s;
}

// Threads per output of a column or row sum over `len` outputs: the block
// splits into S = kSigThreads / C slices of C >= len outputs each; beyond
// 128 outputs C = kSigThreads (S = 1) and each thread sums whole columns or
// rows c, c + C, ...
__device__ __forceinline__ int sig_width(int len) {
  return len <= 32 ? 32 : (len <= 64 ? 64 : (len <= 128 ? 128 : kSigThreads));
}

// Householder bidiagonalisation of the n x n matrix A (row-major, stride lda,
// shared memory; overwritten).  Writes q[k] = d_k^2 and e[k] = f_k^2 (k < n-1)
// with d the diagonal and f the superdiagonal of B.
template <typename T>
__device__ void sig_bidiagonalise(T* A, int lda, int n, T* q, T* e, T* w, T* part, T* red) {
  const int tid = threadIdx.x;
  for (int k = 0; k < n; ++k) {
    // ---- left reflection: x = A[k:, k] -> (d_k, 0, ..., 0)
    T p = T(0);
    for (int i = k + 1 + tid; i < n; i += kSigThreads) p += A[i * lda + k] * A[i * lda + k];
    const T ssl = sig_block_sum(p, red);
    const T x0 = A[k * lda + k];
    T dk = x0;
    if (ssl > T(0) && k + 1 < n) {
      const T alpha = sqrt(x0 * x0 + ssl);
      dk = x0 >= T(0) ? -alpha : alpha;
      const T v0 = x0 - dk;  // v = x - d_k e_1; H = I - beta v v^T
      const T beta = T(-1) / (dk * v0);
      const int len = n - k - 1, C = sig_width(len), S = kSigThreads / C;
      const int c = tid % C, s = tid / C;
      // w_j = beta v^T A[k:, j]
      if (S > 1) {
        const int j = k + 1 + c;
        T acc = T(0);
        if (j < n)
          for (int i = k + s; i < n; i += S) acc += (i == k ? v0 : A[i * lda + k]) * A[i * lda + j];
        part[s * C + c] = acc;
        __syncthreads();
        if (tid < len) {
          T t = T(0);
          for (int u = 0; u < S; ++u) t += part[u * C + tid];
          w[tid] = beta * t;
        }
        __syncthreads();
      } else {  // whole columns: each thread updates only the columns it summed
        for (int cc = c; cc < len; cc += C) {
          const int j = k + 1 + cc;
          T acc = T(0);
          for (int i = k; i < n; ++i) acc += (i == k ? v0 : A[i * lda + k]) * A[i * lda + j];
          w[cc] = beta * acc;
        }
      }
      for (int cc = c; cc < len; cc += C) {
        const int j = k + 1 + cc;
        const T wj = w[cc];
        for (int i = k + s; i < n; i += S) A[i * lda + j] -= (i == k ? v0 : A[i * lda + k]) * wj;
      }
      __syncthreads();
    }
    if (tid == 0) q[k] = dk * dk;
    if (k + 1 >= n) break;
    // ---- right reflection: y = A[k, k+1:] -> (f_k, 0, ..., 0)
    T* red2 = red + kSigWarps;
    p = T(0);
    for (int j = k + 2 + tid; j < n; j += kSigThreads) p += A[k * lda + j] * A[k * lda + j];
    const T ssr = sig_block_sum(p, red2);
    const T y0 = A[k * lda + k + 1];
    T fk = y0;
    if (ssr > T(0)) {
      const T alpha = sqrt(y0 * y0 + ssr);
      fk = y0 >= T(0) ? -alpha : alpha;
      const T u0 = y0 - fk;
      const T beta = T(-1) / (fk * u0);
      const int len = n - k - 1, C = sig_width(len), S = kSigThreads / C;
      const int r = tid % C, s = tid / C;
      // z_i = beta A[i, k+1:] u
      if (S > 1) {
        const int i = k + 1 + r;
        T acc = T(0);
        if (i < n)
          for (int j = k + 1 + s; j < n; j += S) acc += A[i * lda + j] * (j == k + 1 ? u0 : A[k * lda + j]);
        part[s * C + r] = acc;
        __syncthreads();
        if (tid < len) {
          T t = T(0);
          for (int u = 0; u < S; ++u) t += part[u * C + tid];
          w[tid] = beta * t;
        }
      } else {  // whole rows
        for (int rr = r; rr < len; rr += C) {
          const int i = k + 1 + rr;
          T acc = T(0);
          for (int j = k + 1; j < n; ++j) acc += A[i * lda + j] * (j == k + 1 ? u0 : A[k * lda + j]);
          w[rr] = beta * acc;
        }
      }
      __syncthreads();
      // A[k+1:, k+1:] -= z u^T: thread (c, s) walks columns k+1+c, k+1+c+C, ... over the rows of slice s
      for (int cc = r; cc < len; cc += C) {
        const int j = k + 1 + cc;
        const T uj = j == k + 1 ? u0 : A[k * lda + j];
        for (int ii = k + 1 + s; ii < n; ii += S) A[ii * lda + j] -= w[ii - k - 1] * uj;
      }
      __syncthreads();
    }
    if (tid == 0) e[k] = fk * fk;
  }
  __syncthreads();
}

// The same reflections for n <= 32 in warp 0 alone (no block barriers):
// lane j owns column j for the column sums and updates and row j for the
// row sums; the matrix stays in shared memory.
template <typename T>
__device__ void sig_bidiagonalise_warp(T* A, int lda, int n, T* q, T* e, T* w) {
  const int lane = threadIdx.x & 31;
  for (int k = 0; k < n; ++k) {
    // ---- left reflection: x = A[k:, k] -> (d_k, 0, ..., 0)
    T p = lane > k && lane < n ? A[lane * lda + k] * A[lane * lda + k] : T(0);
    for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
    const T x0 = A[k * lda + k];
    T dk = x0;
    if (p > T(0) && k + 1 < n) {
      const T alpha = sqrt(x0 * x0 + p);
      dk = x0 >= T(0) ? -alpha : alpha;
      const T v0 = x0 - dk;
      const T beta = T(-1) / (dk * v0);
      const int j = lane;
      if (j > k && j < n) {
        T acc = v0 * A[k * lda + j];
        for (int i = k + 1; i < n; ++i) acc += A[i * lda + k] * A[i * lda + j];
        const T wj = beta * acc;
        A[k * lda + j] -= v0 * wj;
        for (int i = k + 1; i < n; ++i) A[i * lda + j] -= A[i * lda + k] * wj;
      }
      __syncwarp();
    }
    if (lane == 0) q[k] = dk * dk;
    if (k + 1 >= n) break;
    // ---- right reflection: y = A[k, k+1:] -> (f_k, 0, ..., 0)
    p = lane > k + 1 && lane < n ? A[k * lda + lane] * A[k * lda + lane] : T(0);
    for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
    const T y0 = A[k * lda + k + 1];
    T fk = y0;
    if (p > T(0)) {
      const T alpha = sqrt(y0 * y0 + p);
      fk = y0 >= T(0) ? -alpha : alpha;
      const T u0 = y0 - fk;
      const T beta = T(-1) / (fk * u0);
      if (lane > k && lane < n) {  // z_i = beta A[i, k+1:] u, row i = lane
        const int i = lane;
        T acc = A[i * lda + k + 1] * u0;
        for (int j = k + 2; j < n; ++j) acc += A[i * lda + j] * A[k * lda + j];
        w[i] = beta * acc;
      }
      __syncwarp();
      if (lane > k && lane < n) {  // column j = lane: A[k+1:, j] -= z u_j
        const int j = lane;
        const T uj = j == k + 1 ? u0 : A[k * lda + j];
        for (int i = k + 1; i < n; ++i) A[i * lda + j] -= w[i] * uj;
      }
      __syncwarp();
    }
    if (lane == 0) e[k] = fk * fk;
  }
  __syncwarp();
}

// ------------------------------------------------------------------- dqds --

// dqds on q[0..n-1], e[0..n-2] (warp 0; every lane holds the same scalar
// state).  Writes the eigenvalues of B^T B to lam (any order).  cq / ce hold
// each lane's transform (entry i of lane l at i * kCand + l); stk the split
// stack (3 n doubles).  Returns the number of transforms, or -1 when the
// limit ran out or no shift kept the array positive (NaN input); lam then
// holds the current estimates.
template <typename Num>
__device__ int sig_dqds(typename Num::T* q, typename Num::T* e, int n, double* lam, typename Num::T* cq,
                        typename Num::T* ce, double* stk) {
  using T = typename Num::T;
  const int lane = threadIdx.x & 31;
  constexpr int E = Num::kBits;
  // exact powers of two: lanes 0..30 from 2^-E to 2^-1, lane 31 one (tau = 0)
  const float g = lane == 31 ? 1.0f : ldexpf(1.0f, -E + (lane * (E - 1) + 15) / 30);
  const T tol = Num::from(ldexp(1.0, -2 * E) / 9.0);
  const T zero = Num::from(0.0);
  const int limit = 30 * n + 64;
  int lo = 0, hi = n - 1, depth = 0, transforms = 0;
  T S = zero, dmin = zero, dmin2 = zero;
  bool have = false, failed = false;
  for (;;) {
    if (hi < lo) {
      if (depth == 0) break;
      --depth;
      lo = static_cast<int>(stk[3 * depth]);
      hi = static_cast<int>(stk[3 * depth + 1]);
      S = Num::from(stk[3 * depth + 2]);
      have = false;
      continue;
    }
    if (hi == lo) {
      if (lane == 0) lam[hi] = Num::to_double(Num::add(S, q[hi]));
      --hi;
      continue;
    }
    if (Num::leq(e[hi - 1], Num::mul(tol, Num::add(S, q[hi])))) {  // the last value has converged
      if (lane == 0) lam[hi] = Num::to_double(Num::add(S, q[hi]));
      --hi;
      dmin = dmin2;
      continue;
    }
    // split at the last interior e that no longer couples its neighbours
    const T tS = Num::mul(tol, S);
    int split = -1;
    for (int base = lo; base <= hi - 2; base += 32) {
      const int i = base + lane;
      const unsigned m = __ballot_sync(0xffffffffu, i <= hi - 2 && Num::leq(e[i], tS));
      if (m) split = base + 31 - __clz(m);
    }
    if (split >= 0) {
      if (lane == 0) {
        stk[3 * depth] = lo;
        stk[3 * depth + 1] = split;
        stk[3 * depth + 2] = Num::to_double(S);  // S is a sum of shifts: exact enough in FP64 for a restart
      }
      ++depth;
      lo = split + 1;
      have = false;
      __syncwarp();
      continue;
    }
    if (transforms >= limit) {
      failed = true;
      break;
    }
    // shift estimate: smaller eigenvalue of [[q_{h-1} + e_{h-1}, sqrt(e_{h-1} q_h)], [., q_h]]
    const T a = Num::add(q[hi - 1], e[hi - 1]), c = q[hi];
    const T tr = Num::add(a, c), det = Num::sub(Num::mul(a, c), Num::mul(e[hi - 1], q[hi]));
    T est = zero;
    if (Num::pos(tr)) {
      const T disc = Num::sub(Num::mul(tr, tr), Num::scale(det, 4.0f));
      const T root = Num::nonneg(disc) ? Num::sqrt_(disc) : zero;
      est = Num::div(Num::scale(det, 2.0f), Num::add(tr, root));
    }
    if (have && Num::less(dmin, est)) est = dmin;
    if (!Num::pos(est)) est = zero;
    const T tau = Num::sub(est, Num::scale(est, g));
    // the transform for this lane's shift
    T d = Num::sub(q[lo], tau), dm2 = d;
    bool ok = Num::nonneg(d);
    T ei = e[lo], qn = q[lo + 1];  // loaded one step ahead of the dependent chain
    for (int i = lo; i < hi; ++i) {
      const T ei_next = i + 1 < hi ? e[i + 1] : zero, qn_next = i + 1 < hi ? q[i + 2] : zero;
      const T qh = Num::add(d, ei);
      ok = ok && Num::pos(qh);
      const T t = Num::div(qn, qh);
      cq[(i - lo) * kCand + lane] = qh;
      ce[(i - lo) * kCand + lane] = Num::mul(ei, t);
      if (Num::less(d, dm2)) dm2 = d;
      d = Num::sub(Num::mul(d, t), tau);
      ok = ok && Num::nonneg(d);
      ei = ei_next;
      qn = qn_next;
    }
    cq[(hi - lo) * kCand + lane] = d;
    ++transforms;
    const unsigned good = __ballot_sync(0xffffffffu, ok);
    if (!good) {
      failed = true;
      break;
    }
    const int win = __ffs(good) - 1;  // the largest shift that kept the array positive
    __syncwarp();
    for (int idx = lane; idx <= hi - lo; idx += 32) {
      q[lo + idx] = cq[idx * kCand + win];
      if (idx < hi - lo) e[lo + idx] = ce[idx * kCand + win];
    }
    S = Num::add(S, Num::shfl(tau, win));
    dmin2 = Num::shfl(dm2, win);
    const T dl = Num::shfl(d, win);
    dmin = Num::less(dl, dmin2) ? dl : dmin2;
    have = true;
    __syncwarp();
  }
  if (failed) {  // current estimates for every value not yet converged
    for (;;) {
      for (int i = lo + lane; i <= hi; i += 32) lam[i] = Num::to_double(Num::add(S, q[i]));
      if (depth == 0) break;
      --depth;
      lo = static_cast<int>(stk[3 * depth]);
      hi = static_cast<int>(stk[3 * depth + 1]);
      S = Num::from(stk[3 * depth + 2]);
    }
  }
  __syncwarp();
  return failed ? -1 : transforms;
}

// Shared-memory layout (bytes, 8-byte aligned pieces): region (the matrix
// in T, later the candidates in Num::T), q / e / w (n T each), part
// (kSigThreads T), red (2 kSigWarps T), qq / ee (n Num::T each), lam (n
// doubles), stk (3 n doubles).  The FP32 form needs half the bytes of the
// accurate one, so more CTAs share an SM in a batch.
// The wide form (n > 128) keeps the matrix and the candidates in global
// scratch and only the rest in shared memory.
template <typename T, typename NT>
__host__ __device__ constexpr size_t sig_smem_bytes(int n, bool wide = false) {
  return (wide ? 0 : sig_region_bytes<T, NT>(n)) + sig_al8(sizeof(T) * (3 * n + kSigThreads + 2 * kSigWarps)) +
         sig_al8(sizeof(NT) * 2 * n) + sizeof(double) * 4 * n;
}

// Singular values of the upper triangle of R (n x n, row stride ldr, FP64,
// global memory; the strict lower triangle is not read) into sigma[0..n-1],
// descending.  T: arithmetic of the bidiagonalisation, Num: of dqds.
// *count_out (if not null) receives the number of dqds transforms, or -1
// when dqds stopped early or R holds NaN or Inf (then also
// kStatusNoConvergence in *status, if not null).  gA (n x n T) and gcand
// (2 kCand n NT), both global, hold the matrix and the candidates when not
// null (the wide form); else both live in shared memory.
template <typename T, typename Num>
__device__ void sigma_dqds_body(const double* R, int64_t ldr, int n, double* sigma, int32_t* status,
                                int32_t* count_out, T* gA = nullptr, typename Num::T* gcand = nullptr) {
  using NT = typename Num::T;
  extern __shared__ __align__(16) double sig_sm[];
  const bool wide = gA != nullptr;
  const int lda = wide ? n : sig_lda(n);
  char* base = reinterpret_cast<char*>(sig_sm);
  T* A = wide ? gA : reinterpret_cast<T*>(base);
  char* p1 = base + (wide ? 0 : sig_region_bytes<T, NT>(n));
  T* q = reinterpret_cast<T*>(p1);
  T* e = q + n;
  T* w = e + n;
  T* part = w + n;
  T* red = part + kSigThreads;
  char* p2 = p1 + sig_al8(sizeof(T) * (3 * n + kSigThreads + 2 * kSigWarps));
  NT* qq = reinterpret_cast<NT*>(p2);
  NT* ee = qq + n;
  double* lam = reinterpret_cast<double*>(p2 + sig_al8(sizeof(NT) * 2 * n));
  double* stk = lam + n;
  const int tid = threadIdx.x;
  if (status && (*reinterpret_cast<const volatile int32_t*>(status) & kStatusTimeout)) return;
  // scale by a power of two so that the largest |entry| lies in [1/2, 1)
  double amax = 0.0;
  int bad = 0;
  for (int x = tid; x < n * n; x += kSigThreads) {
    const int i = x / n, j = x % n;
    const double v = j >= i ? R[static_cast<int64_t>(i) * ldr + j] : 0.0;
    bad |= fabs(v) <= DBL_MAX ? 0 : 1;
    amax = fmax(amax, fabs(v));
  }
  if (__syncthreads_or(bad)) {  // NaN or Inf in R
    for (int i = tid; i < n; i += kSigThreads) sigma[i] = NAN;
    if (tid == 0) {
      if (status) set_status(status, kStatusNoConvergence);
      if (count_out) *count_out = -1;
    }
    return;
  }
  for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  // kSigWarps doubles: the start of the matrix region (>= 264 bytes), or part (wide form, T = double)
  double* wmax = wide ? reinterpret_cast<double*>(part) : sig_sm;
  if ((tid & 31) == 0) wmax[tid >> 5] = amax;
  __syncthreads();
  amax = 0.0;
  for (int v = 0; v < kSigWarps; ++v) amax = fmax(amax, wmax[v]);
  __syncthreads();  // every thread has read wmax before the matrix overwrites it
  if (amax == 0.0) {
    for (int i = tid; i < n; i += kSigThreads) sigma[i] = 0.0;
    if (tid == 0 && count_out) *count_out = 0;
    return;
  }
  int ex;
  frexp(amax, &ex);
  const double scale = ldexp(1.0, -ex);
  for (int x = tid; x < n * n; x += kSigThreads) {
    const int i = x / n, j = x % n;
    A[i * lda + j] = static_cast<T>(j >= i ? R[static_cast<int64_t>(i) * ldr + j] * scale : 0.0);
  }
  __syncthreads();
  if (n <= 32) {  // warp 0 alone
    if (tid >= 32) return;
    sig_bidiagonalise_warp<T>(A, lda, n, q, e, w);
  } else {
    sig_bidiagonalise<T>(A, lda, n, q, e, w, part, red);
    if (tid >= 32) return;
  }
  for (int i = tid; i < n; i += 32) {
    qq[i] = Num::from(static_cast<double>(q[i]));
    if (i < n - 1) ee[i] = Num::from(static_cast<double>(e[i]));
  }
  __syncwarp();
  NT* cq = wide ? gcand : reinterpret_cast<NT*>(base);
  const int res = sig_dqds<Num>(qq, ee, n, lam, cq, cq + kCand * n, stk);
  // descending order: rank of each value among all (ties by index)
  const double unscale = ldexp(1.0, ex);
  for (int i = tid; i < n; i += 32) {
    const double li = lam[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double lj = lam[j];
      rank += (lj > li || (lj == li && j < i)) ? 1 : 0;
    }
    sigma[rank] = sqrt(fmax(li, 0.0)) * unscale;
  }
  if (tid == 0) {
    if (res < 0 && status) set_status(status, kStatusNoConvergence);
    if (count_out) *count_out = res;
  }
}

template <typename T, typename Num>
__global__ void __launch_bounds__(kSigThreads) sigma_dqds_kernel(const double* R, int64_t ldr, int n, double* sigma,
                                                                 int32_t* status, int32_t* count_out) {
  pdl_enter();
  sigma_dqds_body<T, Num>(R, ldr, n, sigma, status, count_out);
}

// n in (128, 512]: one CTA, the matrix and candidates in global scratch (accurate form on both paths)
__global__ void __launch_bounds__(kSigThreads) sigma_dqds_wide_kernel(const double* R, int64_t ldr, int n,
                                                                      double* sigma, int32_t* status,
                                                                      int32_t* count_out, double* gA, FF* gcand) {
  pdl_enter();
  sigma_dqds_body<double, FFNum>(R, ldr, n, sigma, status, count_out, gA, gcand);
}

// count matrices R + b * stride, sigma + b * n, info[b] (accurate form)
__global__ void __launch_bounds__(kSigThreads) sigma_dqds_many_kernel(const double* R, int64_t ldr, int64_t stride,
                                                                      int n, double* sigma, int32_t* info) {
  pdl_enter();
  const int b = blockIdx.x;
  sigma_dqds_body<double, FFNum>(R + static_cast<int64_t>(b) * stride, ldr, n, sigma + static_cast<int64_t>(b) * n,
                                 nullptr, info ? info + b : nullptr);
}

template <typename T, typename Num>
__global__ void __launch_bounds__(kSigThreads) sigma_dqds_batched(BatchDev b, BatchJobs J) {
  pdl_enter();
  const int i = J.inst[blockIdx.x];
  const Plan& P = b.plans[i];
  sigma_dqds_body<T, Num>(P.R, P.n, P.n, b.out[i].sigma, &P.hdr->status, &P.hdr->jacobi_sweeps);
}

}  // namespace

size_t sigma_dqds_smem(int n, int mixed) {
  return mixed ? sig_smem_bytes<float, float>(n) : sig_smem_bytes<double, FF>(n);
}
int sigma_dqds_threads() { return kSigThreads; }

cudaError_t launch_sigma_dqds(const Plan& p, const double* R, int64_t ldr, double* sigma, cudaStream_t s) {
  if (p.n > kMaxWidth) {
    // the factorisation's n x n scratch is free by now: G1 holds the matrix
    // (n^2 doubles), G2 the candidates (2 kCand n float-float pairs <= n^2 doubles)
    const size_t smem = sig_smem_bytes<double, FF>(p.n, true);
    cudaError_t err = cudaFuncSetAttribute(sigma_dqds_wide_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    err = pdl_launch(sigma_dqds_wide_kernel, 1, kSigThreads, smem, s, R, ldr, p.n, sigma, &p.hdr->status,
                     &p.hdr->jacobi_sweeps, p.G1, reinterpret_cast<FF*>(p.G2));
    count_launches(1);
    return err != cudaSuccess ? err : cudaGetLastError();
  }
  const size_t smem = sigma_dqds_smem(p.n, p.mixed);
  auto kern = p.mixed ? sigma_dqds_kernel<float, F32Num> : sigma_dqds_kernel<double, FFNum>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  err = pdl_launch(kern, 1, kSigThreads, smem, s, R, ldr, p.n, sigma, &p.hdr->status, &p.hdr->jacobi_sweeps);
  count_launches(1);
  return err != cudaSuccess ? err : cudaGetLastError();
}

cudaError_t launch_sigma_dqds_many(const double* R, int64_t ldr, int64_t stride, int n, int count, double* sigma,
                                   int32_t* info, cudaStream_t s) {
  const size_t smem = sigma_dqds_smem(n, 0);
  cudaError_t err = cudaFuncSetAttribute(sigma_dqds_many_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  err = pdl_launch(sigma_dqds_many_kernel, count, kSigThreads, smem, s, R, ldr, stride, n, sigma, info);
  count_launches(1);
  return err != cudaSuccess ? err : cudaGetLastError();
}

cudaError_t launch_batch_sigma_dqds(const BatchDev& b, const BatchJobs& J, size_t smem, int mixed, cudaStream_t s) {
  if (J.njobs == 0) return cudaSuccess;
  auto kern = mixed ? sigma_dqds_batched<float, F32Num> : sigma_dqds_batched<double, FFNum>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  err = pdl_launch(kern, J.njobs, kSigThreads, smem, s, b, J);  // one CTA per instance
  count_launches(1);
  return err != cudaSuccess ? err : cudaGetLastError();
}

}  // namespace figaro
