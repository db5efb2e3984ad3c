// Small dense n x n steps of CholeskyQR2 and the singular values.  One CTA
// per instance (n <= 128): for n <= 32 the matrix lives in registers (the
// register-resident forms below), above in shared memory.
//
//  * chol_first:  R1 = chol(G1), semi-definite: a pivot below
//                 rank_tol * G1_kk marks column k as dependent (zero row);
//                 W = R1^{-1} on the independent columns.
//  * chol_second: R2 = chol(G2) on the same columns, R = R2 R1 in FP64.  The
//                 diagonal is positive, so R has the sign convention of
//                 Section 1 (R is the Cholesky factor of J^T J).
//  * jacobi:      one-sided (Hestenes) Jacobi on the columns of R (Section 3:
//                 the singular values of J are those of R), parallel
//                 round-robin ordering, one thread group per column pair.
//
// Precision.  Plain path: every step in FP64.  Mixed path: the two Cholesky
// factorisations and the inverse run in FP32 -- R1 is only a preconditioner
// (its rounding is removed by the second pass, and W is the exact inverse
// used to form Q), and G2 = I + O(u) so R2 = chol(G2) in FP32 has an absolute
// error of a few FP32 ulps -- while R = R2 R1 is formed in extended precision
// (FP64; float-float for n <= 32); the Jacobi sweeps run in FP32 accumulating
// V and each singular value is then the Rayleigh quotient ||R v_j|| / ||v_j||
// in extended precision, whose error is second order in the FP32 error of
// v_j.  FP64 is slow on this GPU (about 2 FMA per SM per clock, 64 cycles of
// latency, hundreds per sqrt or divide), so the FP64 pivots use an FP32 seed
// refined by two Newton steps for 1/sqrt(d), dot products are split across
// lanes, and the n <= 32 forms use float-float (exact FMA products,
// compensated sums) instead.
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace figaro {
namespace {


// In-place semi-definite Cholesky of the n x n matrix A (shared memory,
// row-major, upper triangle used).  act[k]: columns marked 0 on entry stay
// dependent.  On return the upper triangle holds the factor R.  Every thread
// evaluates the pivot of step k itself (same operands, same result), so a
// step needs one barrier; thread (r, c) of the 2D map updates the trailing
// entries (i, j), k < i <= j, with i = r (mod rows) and j = c (mod 32).
template <typename T>
__device__ void chol_inplace(T* A, int n, const T* diag0, int32_t* act, T tol, T* y, int32_t* status) {
  const int c0 = threadIdx.x & 31, r0 = threadIdx.x >> 5, rstep = blockDim.x >> 5;
  for (int k = 0; k < n; ++k) {
    const T d = A[k * n + k];
    const int was = act[k];
    int ok = was;
    if (!isfinite(d)) ok = 0;
    if (!(d > tol * diag0[k]) || !(diag0[k] > T(0))) ok = 0;
    const bool dropped = was && !ok && isfinite(d) && diag0[k] > T(0);
    const T yk = ok ? rsqrt_pivot(d) : T(0);
    if (yk != T(0)) {
      const T y2 = yk * yk;
      for (int i = k + 1 + r0; i < n; i += rstep) {
        const T aki = A[k * n + i] * y2;
        for (int j = i + ((c0 - i) & 31); j < n; j += 32) A[i * n + j] -= aki * A[k * n + j];
      }
    }
    if (threadIdx.x == 0) {
      if (!isfinite(d)) set_status(status, kStatusNotSpd);
      if (dropped) note_dropped(status, k);
      act[k] = ok;
      y[k] = yk;
    }
    __syncthreads();
  }
  // scale rows: R[k][j] = A[k][j] y[k] for j >= k (R[k][k] = sqrt(d_k))
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e - i * n;
    if (j >= i) A[e] *= y[i];
  }
  __syncthreads();
}

// W = R^{-1} (upper triangular, R in A) into a separate buffer W: column j
// by back substitution, W[j][j] = 1 / R[j][j], W[i][j] = -(sum_{k=i+1..j}
// R[i][k] W[k][j]) / R[i][i] for i < j; one thread per column (its own
// column of W only, R read-only), no barriers inside.
template <typename T>
__device__ void tri_inverse_cols(const T* __restrict__ A, T* __restrict__ W, int n, const int32_t* act) {
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const bool aj = act[j] != 0;
    for (int i = 0; i < n; ++i) W[i * n + j] = T(0);
    if (!aj) continue;
    W[j * n + j] = T(1) / A[j * n + j];
    for (int i = j - 1; i >= 0; --i) {
      if (!act[i]) continue;
      T s0 = T(0), s1 = T(0);
      int k = i + 1;
      for (; k + 1 <= j; k += 2) {
        s0 += A[i * n + k] * W[k * n + j];
        s1 += A[i * n + k + 1] * W[(k + 1) * n + j];
      }
      if (k <= j) s0 += A[i * n + k] * W[k * n + j];
      W[i * n + j] = -(s0 + s1) / A[i * n + i];
    }
  }
  __syncthreads();
}

// Warp-cooperative in-place inverse of the upper-triangular R (n x n, shared
// memory) on the independent columns: column j of W needs W's leading j x j
// block and column j of R only.
template <typename T>
__device__ void tri_inverse_inplace(T* A, int n, const int32_t* act, T* x) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < n; ++j) {
    const bool aj = act[j] != 0;
    for (int i = warp; i < j; i += nw) {
      T s = T(0);
      if (aj && act[i])
        for (int k = i + lane; k < j; k += 32) s += A[i * n + k] * A[k * n + j];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) x[i] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) A[j * n + j] = aj ? T(1) / A[j * n + j] : T(0);
    __syncthreads();
    const T wjj = A[j * n + j];
    for (int i = threadIdx.x; i < j; i += blockDim.x) A[i * n + j] = (aj && act[i]) ? -x[i] * wjj : T(0);
    __syncthreads();
  }
}

// Shift of the shifted CholeskyQR3 (Fukaya et al., SIAM J. Sci. Comput. 42
// (2020)): shift_rel times the trace of G, added to the non-zero diagonal
// entries, so that the factorisation of an ill-conditioned G succeeds.
__device__ __forceinline__ double gram_shift(const double* G, int n, double shift_rel) {
  if (!(shift_rel > 0.0)) return 0.0;
  double tr = 0.0;
  for (int k = 0; k < n; ++k) tr += G[k * n + k];
  return shift_rel * tr;
}

// First factorisation (n <= 128): R1 = chol(G1 + shift) and W = R1^{-1}.
// from_r: G holds an upper-triangular R instead (the shifted CholeskyQR3's
// second factor); R1 = R and W = R^{-1} on the columns with R_kk != 0.
template <typename T, bool kSmall>
__device__ __forceinline__ void chol_first_body(const double* G, int n, double tol, double* R1, double* W, float* Wf,
                                                int32_t* active, int32_t* status, double shift_rel, int from_r) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* A = reinterpret_cast<T*>(smraw);  // n x n
  T* diag0 = A + n * n;
  T* y = diag0 + n;
  T* x = y + n;
  int32_t* act = reinterpret_cast<int32_t*>(x + n);
  const double shift = from_r ? 0.0 : gram_shift(G, n, shift_rel);
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    const double g = G[e];
    A[e] = static_cast<T>(i == j && g > 0.0 ? g + shift : g);
  }
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const double g = G[k * n + k];
    diag0[k] = static_cast<T>(g > 0.0 ? g + shift : g);
    act[k] = from_r ? (g != 0.0) : 1;
  }
  __syncthreads();
  if (!from_r) chol_inplace<T>(A, n, diag0, act, static_cast<T>(tol), y, status);
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    R1[e] = (j >= i && act[i]) ? (from_r ? G[e] : static_cast<double>(A[e])) : 0.0;
  }
  for (int k = threadIdx.x; k < n; k += blockDim.x) active[k] = act[k];
  __syncthreads();
  if constexpr (kSmall) {  // a second n x n buffer follows the work arrays
    T* Wb = reinterpret_cast<T*>(act + n + ((4 - (n & 3)) & 3));
    tri_inverse_cols<T>(A, Wb, n, act);
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) A[e] = Wb[e];
    __syncthreads();
  } else {
    tri_inverse_inplace<T>(A, n, act, x);
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    // dependent columns pass through the second pass unchanged (identity
    // block), so their coupling to the independent ones is measured there
    double w = (j >= i) ? static_cast<double>(A[e]) : 0.0;
    if (i == j && !act[i]) w = 1.0;
    if (sizeof(T) == 4) {
      // the value both Gram engines use exactly: hi (TF32) + lo rounded to TF32
      const float v = static_cast<float>(w);
      const float h = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
      const float l = __uint_as_float((__float_as_uint(v - h) + 0x1000u) & 0xFFFFE000u);
      w = static_cast<double>(h + l);
    }
    W[e] = w;
    Wf[e] = static_cast<float>(w);
  }
}

template <typename T, bool kSmall>
__global__ void __launch_bounds__(1024) chol_first_kernel(const double* G, int n, double tol, double* R1, double* W, float* Wf,
                                  int32_t* active, int32_t* status, double shift_rel, int from_r) {
  pdl_enter();
  chol_first_body<T, kSmall>(G, n, tol, R1, W, Wf, active, status, shift_rel, from_r);
}

// Upper-triangular product C = A B on n x n row-major matrices, one thread
// per output, two partial sums to shorten the FP64 dependency chain.
template <typename TA, typename TB>
__device__ __forceinline__ double upper_dot(const TA* A, const TB* B, int n, int i, int j) {
  double s0 = 0.0, s1 = 0.0;
  int k = i;
  for (; k + 1 <= j; k += 2) {
    s0 += static_cast<double>(A[i * n + k]) * static_cast<double>(B[k * n + j]);
    s1 += static_cast<double>(A[i * n + k + 1]) * static_cast<double>(B[(k + 1) * n + j]);
  }
  if (k <= j) s0 += static_cast<double>(A[i * n + k]) * static_cast<double>(B[k * n + j]);
  return s0 + s1;
}

// hi + lo += x y exactly up to the final rounding of lo (the product's
// rounding error recovered by an FMA, the sum by TwoSum).
__device__ __forceinline__ void ff_fma(float& hi, float& lo, float x, float y) {
  const float p = x * y;
  const float e = fmaf(x, y, -p);
  float s, t;
  two_sum(hi, p, s, t);
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(t, e));
}

// Offset of row i of a packed upper triangle (rows i..n-1 of lengths n - i).
__device__ __forceinline__ int tri_row(int n, int i) { return i * n - (i * (i - 1)) / 2; }

// Mixed-path second factorisation and R for 32 < n <= 128 (one CTA): as the
// n <= 32 form, E = I - W R1 in float-float from the exact FP32 values of W
// and R1, X = R1 + R1 E kept as the pair (R1 masked, the FP32 correction
// R1 E), R = R2 X in float-float.  Shared memory: A (n x n, G2 then R2) and
// three packed upper triangles (R1 then the X head, W then the X correction,
// E).  Xg receives X in FP64, as the FP64 form writes it.
__device__ __forceinline__ void chol_second_ff_body(const double* G2, int n, double tol, const double* R1,
                                                    const float* Wf, const int32_t* active, double* Xg, double* R,
                                                    double* R_out, int64_t ldr, int32_t* status) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int nt = n * (n + 1) / 2;
  float* A = reinterpret_cast<float*>(smraw);
  float* diag0 = A + n * n;
  float* y = diag0 + n;
  int32_t* act = reinterpret_cast<int32_t*>(y + n);
  float* tX = reinterpret_cast<float*>(act + n);  // R1, then X's head
  float* tL = tX + nt;                              // W, then X's correction
  float* tE = tL + nt;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) A[e] = static_cast<float>(G2[e]);
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    diag0[k] = static_cast<float>(G2[k * n + k]);
    act[k] = active[k];
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e - (e / n) * n;
    if (j < i) continue;
    const int t = tri_row(n, i) + (j - i);
    tX[t] = static_cast<float>(R1[e]);  // (exact: R1 holds FP32 values)
    tL[t] = Wf[e];
  }
  __syncthreads();
  // E = I - W R1 on the independent columns
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e - (e / n) * n;
    if (j < i) continue;
    float ev = 0.f;
    if (act[i] && act[j]) {
      float hi = 0.f, lo = 0.f;
      const int wi = tri_row(n, i) - i;  // W[i][k] = tL[wi + k]
      int kj = tri_row(n, i) + (j - i);  // R1[k][j], k = i..j
      for (int k = i; k <= j; ++k) {
        ff_fma(hi, lo, tL[wi + k], tX[kj]);
        kj += n - k - 1;
      }
      float t0, t1;
      two_sum(i == j ? 1.f : 0.f, -hi, t0, t1);
      ev = __fadd_rn(t0, __fadd_rn(t1, -lo));
    }
    tE[tri_row(n, i) + (j - i)] = ev;
  }
  __syncthreads();
  // the correction R1 E (FP32: it is ~1e-7 of R1) into W's triangle
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e - (e / n) * n;
    if (j < i) continue;
    float c = 0.f;
    if (act[i] && act[j]) {
      const int ri = tri_row(n, i) - i;
      int kj = tri_row(n, i) + (j - i);
      for (int k = i; k <= j; ++k) {
        c = fmaf(tX[ri + k], tE[kj], c);
        kj += n - k - 1;
      }
    }
    tL[tri_row(n, i) + (j - i)] = c;
  }
  __syncthreads();
  // X's head: R1 on the independent columns, the identity on the dependent diagonal
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e - (e / n) * n;
    double xd = 0.0;
    if (j >= i) {
      const int t = tri_row(n, i) + (j - i);
      float x = (act[i] && act[j]) ? tX[t] : 0.f;
      if (i == j && !act[i]) x = 1.f;
      tX[t] = x;
      xd = static_cast<double>(x) + static_cast<double>(tL[t]);
    }
    Xg[e] = xd;
  }
  __syncthreads();
  chol_inplace<float>(A, n, diag0, act, static_cast<float>(tol), y, status);
  if (threadIdx.x == 0) {
    int dep = 0;
    for (int k = 0; k < n; ++k) dep += act[k] ? 0 : 1;
    header_of(status)->dep_cols = dep;
  }
  // R = R2 X (both upper triangular); rows of dependent columns are zero
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e - (e / n) * n;
    double r = 0.0;
    if (j >= i && act[i]) {
      float hi = 0.f, lo = 0.f;
      int kj = tri_row(n, i) + (j - i);
      for (int k = i; k <= j; ++k) {
        const float r2 = A[i * n + k];
        ff_fma(hi, lo, r2, tX[kj]);
        lo = fmaf(r2, tL[kj], lo);
        kj += n - k - 1;
      }
      r = static_cast<double>(hi) + static_cast<double>(lo);
    }
    R[e] = r;
    if (R_out) R_out[static_cast<int64_t>(i) * ldr + j] = r;
  }
}

template <typename T>
__device__ __forceinline__ void chol_second_body(const double* G2, int n, double tol, const double* R1, const double* Wd,
                                                 const int32_t* active, int refine, double* Xg, double* R,
                                                 double* R_out, int64_t ldr, int32_t* status) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* A = reinterpret_cast<T*>(smraw);
  T* diag0 = A + n * n;
  T* y = diag0 + n;
  int32_t* act = reinterpret_cast<int32_t*>(y + n);
  double* E = reinterpret_cast<double*>(smraw + ((sizeof(T) * (static_cast<size_t>(n) * n + 2 * n) +
                                                  sizeof(int32_t) * n + 15) & ~static_cast<size_t>(15)));
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) A[e] = static_cast<T>(G2[e]);
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    diag0[k] = static_cast<T>(G2[k * n + k]);
    act[k] = active[k];
  }
  __syncthreads();
  // X = W^{-1} = blockdiag(R1 on the independent columns, I on the others)
  if (refine) {
    // Q was formed with W, so the consistent factor is R2 W^{-1}; one Newton
    // step X = R1 + R1 (I - W R1) squares the relative error of R1 as an
    // inverse of W (FP32 level -> FP64 level)
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int i = e / n, j = e % n;
      E[e] = (j >= i && act[i] && act[j]) ? (i == j ? 1.0 : 0.0) - upper_dot(Wd, R1, n, i, j) : 0.0;
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    double x = 0.0;
    if (j >= i && act[i] && act[j]) x = R1[e] + (refine ? upper_dot(R1, E, n, i, j) : 0.0);
    if (i == j && !act[i]) x = 1.0;
    Xg[e] = x;
  }
  __threadfence_block();
  __syncthreads();
  const double* X = Xg;
  chol_inplace<T>(A, n, diag0, act, static_cast<T>(tol), y, status);
  if (threadIdx.x == 0) {
    int dep = 0;
    for (int k = 0; k < n; ++k) dep += act[k] ? 0 : 1;
    header_of(status)->dep_cols = dep;
  }
  // R = R2 X (both upper triangular) in FP64; rows of dependent columns are zero
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    const double s = (j >= i && act[i]) ? upper_dot(A, X, n, i, j) : 0.0;
    R[e] = s;
    if (R_out) R_out[static_cast<int64_t>(i) * ldr + j] = s;
  }
}

// Shared memory of the one-CTA second factorisation: the float-float form
// (mixed path) or the FP64 one.
__host__ __device__ inline size_t chol_second_smem(int n, bool mixed) {
  if (mixed)
    return (sizeof(float) * (static_cast<size_t>(n) * n + 2 * n) + sizeof(int32_t) * n +
            3 * sizeof(float) * static_cast<size_t>(n) * (n + 1) / 2 + 15) & ~size_t(15);
  return (sizeof(double) * (static_cast<size_t>(n) * n + 2 * n) + sizeof(int32_t) * n + 15) & ~size_t(15);
}

template <typename T, bool kSmall>
__global__ void __launch_bounds__(1024) chol_second_kernel(const double* G2, int n, double tol, const double* R1, const double* Wd,
                                   const float* Wf, const int32_t* active, int refine, double* Xg, double* R,
                                   double* R_out, int64_t ldr, int32_t* status) {
  pdl_enter();
  if constexpr (sizeof(T) == 4) {
    if (refine) {
      chol_second_ff_body(G2, n, tol, R1, Wf, active, Xg, R, R_out, ldr, status);
      return;
    }
  }
  chol_second_body<T>(G2, n, tol, R1, Wd, active, refine, Xg, R, R_out, ldr, status);
}

template <typename T>
__device__ __forceinline__ T group_sum(T v, int width) {
  for (int o = width >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, width);
  return v;
}

// Rotation (c, s) that makes columns p and q orthogonal, from their 2 x 2
// Gram [al ga; ga be]: t = sign(z) / (|z| + sqrt(1 + z^2)), z = (be - al) / (2 ga).
// (FP32 sweeps: the rotations only steer the iteration, the singular values
// come from FP64 Rayleigh quotients, so fast approximate intrinsics suffice.)
__device__ __forceinline__ void rotation(float al, float be, float ga, float& c, float& s) {
  const float z = __fdividef(be - al, 2.f * ga);
  const float az = fabsf(z);
  const float q = 1.f + z * z;
  const float t = az > 1e18f ? __fdividef(0.5f, z) : copysignf(__fdividef(1.f, az + q * rsqrtf(q)), z);
  c = rsqrtf(1.f + t * t);
  s = c * t;
}
__device__ __forceinline__ void rotation(double al, double be, double ga, double& c, double& s) {
  const double z = (be - al) / (2.0 * ga);
  const double t = (z >= 0.0 ? 1.0 : -1.0) / (fabs(z) + sqrt(1.0 + z * z));
  c = 1.0 / sqrt(1.0 + t * t);
  s = c * t;
}

// Shared memory of the one-CTA Jacobi before the bf16 tails of R (mixed path):
// U and V (np x n each with V), sigma and the column norms (np doubles each),
// R in FP64 when V is kept and n <= 64, the pairing table.
__host__ __device__ inline size_t jacobi_smem_base(int n, int es, bool with_v) {
  const size_t np = static_cast<size_t>(n + (n & 1));
  size_t b = es * np * n * (with_v ? 2 : 1) + 2 * sizeof(double) * np;
  if (with_v && n <= 64) b += sizeof(double) * static_cast<size_t>(n) * n;
  return b + sizeof(short2) * (np - 1) * (np / 2);
}
// the bf16 tails of R (n x n) follow at a 16-byte boundary (mixed path, V kept)
__host__ __device__ inline size_t jacobi_rlo_offset(int n, int es) { return (jacobi_smem_base(n, es, true) + 15) & ~size_t(15); }
__host__ __device__ inline size_t jacobi_smem(int n, int es, bool with_v) {
  return with_v && es == 4 ? jacobi_rlo_offset(n, es) + 2 * static_cast<size_t>(n) * n : jacobi_smem_base(n, es, with_v);
}

// One-sided Jacobi.  U (and V) column-major in shared memory; LPP lanes per
// column pair (32 / LPP pairs per warp), NPL rows of each column per lane;
// the round-robin pairing is tabulated once.  A pair is rotated while
// |u_p.u_q|^2 > tol^2 |u_p|^2 |u_q|^2.  With several pairs per warp, the
// pair groups of a warp visit their rows in rotated order (group gw starts
// at row block gw), so that at each step they read different banks.
template <typename T, bool kWithV, int NPL, int LPP>
__device__ __forceinline__ void jacobi_body(const double* R, int64_t ldr, int n, int max_sweeps, double tol_in,
                                            double* sigma, int32_t* status, int32_t* sweeps_out) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int np = n + (n & 1);  // even number of columns (one zero column if n is odd)
  const int npairs = np / 2, rounds = np - 1;
  T* U = reinterpret_cast<T*>(smraw);
  T* V = U + static_cast<int64_t>(np) * n;
  double* sig = reinterpret_cast<double*>(smraw + sizeof(T) * static_cast<size_t>(np) * n * (kWithV ? 2 : 1));
  double* unrm = sig + np;  // column norms of the converged U
  double* Rs = unrm + np;   // R (FP64) for the Rayleigh quotients, when it fits
  short2* pairs = reinterpret_cast<short2*>(Rs + ((kWithV && n <= 64) ? n * n : 0));
  const bool r_in_smem = kWithV && n <= 64;
  __shared__ T s_fro;
  for (int e = threadIdx.x; e < np * n; e += blockDim.x) {
    const int c = e / n, r = e % n;
    U[e] = c < n ? static_cast<T>(R[static_cast<int64_t>(r) * ldr + c]) : T(0);
    if (kWithV) V[e] = (c == r) ? T(1) : T(0);
  }
  if (r_in_smem)
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) Rs[e] = R[static_cast<int64_t>(e / n) * ldr + e % n];
  for (int e = threadIdx.x; e < rounds * npairs; e += blockDim.x) {
    const int round = e / npairs, g = e % npairs;
    int p = g == 0 ? round : (round + g) % (np - 1);
    int q = g == 0 ? np - 1 : (round - g + (np - 1)) % (np - 1);
    if (p > q) {
      const int t = p;
      p = q;
      q = t;
    }
    pairs[e] = make_short2(static_cast<short>(p), static_cast<short>(q));
  }
  __syncthreads();
  const T tol2 = static_cast<T>(tol_in) * static_cast<T>(tol_in);
  // columns whose squared norm is below (n eps)^2 ||R||_F^2 are rounding
  // noise of a rank-deficient R: they take no part in rotations
  if (threadIdx.x < 32) {
    T f = 0;
    for (int e = threadIdx.x; e < np * n; e += 32) f += U[e] * U[e];
    for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
    if (threadIdx.x == 0) s_fro = f;
  }
  __syncthreads();
  // columns below n eps64 ||R||_F are rounding noise of a rank-deficient R
  // and take no part in rotations (the FP64 unit even for FP32 sweeps: FP32
  // dot products keep their relative accuracy under column scaling, so the
  // legitimately small columns of a graded R must keep rotating)
  const double eps64 = 1.1102230246251565e-16;
  const T negligible = static_cast<T>((n * eps64) * (n * eps64) * static_cast<double>(s_fro));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  constexpr int kPPW = 32 / LPP;  // pairs per warp
  const int sub = lane % LPP, gw = lane / LPP;
  int sweep = 0;
  bool converged = false;
  for (; sweep < max_sweeps && !converged; ++sweep) {
    int any = 0;
    for (int round = 0; round < rounds; ++round) {
      for (int g0 = warp * kPPW; g0 < npairs; g0 += nwarps * kPPW) {
        const int g = g0 + gw;
        const bool live = g < npairs;  // (lanes of a missing pair still join the shuffles)
        const short2 pq = live ? pairs[round * npairs + g] : make_short2(0, 0);
        T* up = U + static_cast<int64_t>(pq.x) * n;
        T* uq = U + static_cast<int64_t>(pq.y) * n;
        T x[NPL], y[NPL];
        T al = 0, be = 0, ga = 0;
#pragma unroll
        for (int i = 0; i < NPL; ++i) {
          const int r = sub + LPP * ((i + gw) % NPL);
          x[i] = (live && r < n) ? up[r] : T(0);
          y[i] = (live && r < n) ? uq[r] : T(0);
          al += x[i] * x[i];
          be += y[i] * y[i];
          ga += x[i] * y[i];
        }
#pragma unroll
        for (int o = LPP / 2; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o, LPP);
          be += __shfl_xor_sync(0xffffffffu, be, o, LPP);
          ga += __shfl_xor_sync(0xffffffffu, ga, o, LPP);
        }
        if (live && al > negligible && be > negligible && ga * ga > tol2 * al * be) {
          T c, s;
          rotation(al, be, ga, c, s);
#pragma unroll
          for (int i = 0; i < NPL; ++i) {
            const int r = sub + LPP * ((i + gw) % NPL);
            if (r < n) {
              up[r] = c * x[i] - s * y[i];
              uq[r] = s * x[i] + c * y[i];
            }
          }
          if (kWithV) {
            T* vp = V + static_cast<int64_t>(pq.x) * n;
            T* vq = V + static_cast<int64_t>(pq.y) * n;
#pragma unroll
            for (int i = 0; i < NPL; ++i) {
              const int r = sub + LPP * ((i + gw) % NPL);
              if (r < n) {
                const T xv = vp[r], yv = vq[r];
                vp[r] = c * xv - s * yv;
                vq[r] = s * xv + c * yv;
              }
            }
          }
          any = 1;
        }
      }
      any = __syncthreads_or(any);
    }
    converged = any == 0;
  }
  if (!converged && threadIdx.x == 0) set_status(status, kStatusNoConvergence);
  if (threadIdx.x == 0 && sweeps_out) *sweeps_out = sweep;
  // singular values
  if (kWithV) {
    // ||u_j|| in FP64 from the FP32 columns (kept for the smallest values: the
    // Rayleigh quotient below has an error of order tol sigma_max when
    // sigma_j is near zero, the column norm one of a few FP32 ulps)
    for (int j = warp; j < n; j += nwarps) {
      double un = 0.0;
      const T* uj = U + static_cast<int64_t>(j) * n;
      for (int i = lane; i < n; i += 32) {
        const double u = static_cast<double>(uj[i]);
        un += u * u;
      }
      for (int o = 16; o > 0; o >>= 1) un += __shfl_xor_sync(0xffffffffu, un, o);
      if (lane == 0) unrm[j] = sqrt(un);
    }
    __syncthreads();
    if constexpr (sizeof(T) == 4) {
      // sigma_j^2 = sum_i (R v_j)_i^2 / ||v_j||^2 with (R v_j)_i in
      // float-float: R is split once into FP32 heads (in V's storage) and
      // bf16 tails (their product with v only feeds the low word), V^T goes
      // into U's storage (U and V are no longer needed), so that a warp's
      // lanes (consecutive j) read consecutive words while R[i][k] is one
      // broadcast; warp w takes the 32 columns of block w % jb and the rows
      // i = w / jb (mod ig).  The groups' sums meet in the pairing table's
      // storage.  (FP64 arithmetic is slow on this GPU: one FP64 operation per
      // entry of R, none per product.)
      float* VT = reinterpret_cast<float*>(U);
      for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int j = e / n, k = e - (e / n) * n;
        VT[k * n + j] = V[e];
      }
      __syncthreads();
      float* Rh = reinterpret_cast<float*>(V);
      uint16_t* Rl = reinterpret_cast<uint16_t*>(smraw + jacobi_rlo_offset(n, static_cast<int>(sizeof(T))));
      for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, k = e - (e / n) * n;
        const double r = k >= i ? R[static_cast<int64_t>(i) * ldr + k] : 0.0;
        const float rh = static_cast<float>(r);
        Rh[e] = rh;
        Rl[e] = static_cast<uint16_t>(__float_as_uint(static_cast<float>(r - static_cast<double>(rh))) >> 16);
      }
      for (int j = threadIdx.x; j < n; j += blockDim.x) {  // ||v_j||^2, kept in sig until the end
        double den = 0.0;
        for (int k = 0; k < n; ++k) {
          const double v = static_cast<double>(VT[k * n + j]);
          den += v * v;
        }
        sig[j] = den;
      }
      double* gsum = reinterpret_cast<double*>(pairs);
      const int jb = (n + 31) / 32;
      const int ig = nwarps / jb > 0 ? nwarps / jb : 1;
      __syncthreads();
      for (int w = warp; w < jb * ig; w += nwarps) {
        const int j = (w % jb) * 32 + lane, grp = w / jb;
        if (j >= n) continue;
        double num = 0.0;
        for (int i = grp; i < n; i += ig) {
          float hi = 0.f, lo = 0.f;
          for (int k = i; k < n; ++k) {
            const float v = VT[k * n + j];
            ff_fma(hi, lo, Rh[i * n + k], v);
            lo = fmaf(__uint_as_float(static_cast<uint32_t>(Rl[i * n + k]) << 16), v, lo);
          }
          const double yd = static_cast<double>(hi) + static_cast<double>(lo);
          num += yd * yd;
        }
        gsum[grp * n + j] = num;
      }
      __syncthreads();
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double num = 0.0;
        for (int g = 0; g < ig; ++g) num += gsum[g * n + j];
        const double den = sig[j];
        sig[j] = den > 0.0 ? sqrt(num / den) : 0.0;
      }
      __syncthreads();
    } else {
      for (int j = warp; j < n; j += nwarps) sig[j] = 0.0;
      // sigma_j^2 = sum_i (R v_j)_i^2 / ||v_j||^2 in FP64, one thread per (i, j).
      // U is no longer needed: its storage (np * n floats = np * n / 2 doubles)
      // holds the squared terms for np / 2 rows i at a time.
      double* acc = reinterpret_cast<double*>(U);
      const int ipass = np / 2;
      for (int i0 = 0; i0 < n; i0 += ipass) {
        const int i1 = i0 + ipass < n ? i0 + ipass : n;
        __syncthreads();
        for (int e = threadIdx.x; e < (i1 - i0) * n; e += blockDim.x) {
          const int j = e / (i1 - i0), i = i0 + e % (i1 - i0);
          const T* vj = V + static_cast<int64_t>(j) * n;
          double y0 = 0.0, y1 = 0.0;
          int k = i;
          if (r_in_smem) {
            for (; k + 1 < n; k += 2) {
              y0 += Rs[i * n + k] * static_cast<double>(vj[k]);
              y1 += Rs[i * n + k + 1] * static_cast<double>(vj[k + 1]);
            }
            if (k < n) y0 += Rs[i * n + k] * static_cast<double>(vj[k]);
          } else {
            for (; k < n; ++k) y0 += R[static_cast<int64_t>(i) * ldr + k] * static_cast<double>(vj[k]);
          }
          const double yy = y0 + y1;
          acc[e] = yy * yy;
        }
        __syncthreads();
        for (int j = warp; j < n; j += nwarps) {
          double num = 0.0;
          for (int i = lane; i < i1 - i0; i += 32) num += acc[j * (i1 - i0) + i];
          for (int o = 16; o > 0; o >>= 1) num += __shfl_xor_sync(0xffffffffu, num, o);
          if (lane == 0) sig[j] += num;
        }
      }
      __syncthreads();
      for (int j = warp; j < n; j += nwarps) {
        double den = 0.0;
        const T* vj = V + static_cast<int64_t>(j) * n;
        for (int i = lane; i < n; i += 32) {
          const double v = static_cast<double>(vj[i]);
          den += v * v;
        }
        for (int o = 16; o > 0; o >>= 1) den += __shfl_xor_sync(0xffffffffu, den, o);
        if (lane == 0) sig[j] = den > 0.0 ? sqrt(sig[j] / den) : 0.0;
      }
      __syncthreads();
    }
    double umax = 0.0;
    for (int k = 0; k < n; ++k) umax = unrm[k] > umax ? unrm[k] : umax;
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x)
      if (unrm[j] < 1e-3 * umax) sig[j] = unrm[j];
  } else {
    for (int j = warp; j < n; j += nwarps) {
      double num = 0.0;
      const T* uj = U + static_cast<int64_t>(j) * n;
      for (int i = lane; i < n; i += 32) {
        const double u = static_cast<double>(uj[i]);
        num += u * u;
      }
      for (int o = 16; o > 0; o >>= 1) num += __shfl_xor_sync(0xffffffffu, num, o);
      if (lane == 0) sig[j] = sqrt(num);
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double v = sig[j];
    int rank = 0;
    for (int k = 0; k < n; ++k) {
      const double w = sig[k];
      rank += (w > v) || (w == v && k < j);
    }
    sigma[rank] = v;
  }
}

template <typename T, bool kWithV, int NPL, int LPP>
__global__ void __launch_bounds__(512) jacobi_kernel(const double* R, int64_t ldr, int n, int max_sweeps, double tol_in, double* sigma,
                              int32_t* status, int32_t* sweeps_out) {
  pdl_enter();
  jacobi_body<T, kWithV, NPL, LPP>(R, ldr, n, max_sweeps, tol_in, sigma, status, sweeps_out);
}

__host__ __device__ inline double dense_tol(const Plan& p) {
  return p.rank_tol > 0 ? p.rank_tol : (p.mixed ? 1e-5 : 1e-13);
}
__host__ __device__ inline double jacobi_tol(const Plan& p) {
  return p.mixed ? 1e-5 : 4.0 * p.n * 1.1102230246251565e-16;
}

// ---- register-resident forms for n <= 32 (one column per lane) ----------
//
// At these widths a barrier per elimination step or per rotation round
// dominates, so the work per step must be short: column c of the n x n
// matrix is held by lane c, and row i by warp i mod 8 (register i / 8) for
// the factorisations, or by warp i / (32 / JW) for the Jacobi sweeps.
constexpr int kSmallN = 32;
constexpr int kJacobiLPP = 8;  // lanes per column pair of the shared-memory Jacobi (4 pairs per warp)
constexpr int kC8Warps = 8;  // warps of the small factorisations (rows i = warp + 8 s, s < 4)
constexpr int kC8Threads = 32 * kC8Warps;

template <typename T>
__device__ __forceinline__ T row_reg(const T (&a)[4], int s) {  // a[s], s warp-uniform
  return s == 0 ? a[0] : (s == 1 ? a[1] : (s == 2 ? a[2] : a[3]));
}
template <typename T>
__device__ __forceinline__ void set_row_reg(T (&a)[4], int s, T v) {
  a[0] = s == 0 ? v : a[0];
  a[1] = s == 1 ? v : a[1];
  a[2] = s == 2 ? v : a[2];
  a[3] = s == 3 ? v : a[3];
}

// Semi-definite Cholesky on the 8-warp layout, in place: on entry a[s] =
// A[warp + 8 s][lane] (upper triangle used), on return R (zero below the
// diagonal and in the rows of dependent columns).  Bit k of `mask`: column
// k independent (on entry and on return).  Step k: warp k mod 8 forms row k
// of R from its own registers (the pivot A[k][k] comes from lane k) and
// posts it; after one barrier every thread takes R[k][i] R[k][lane] off its
// rows i > k.  The posted rows alternate between two buffers, so one
// barrier per step suffices.
template <typename T>
__device__ __forceinline__ uint32_t chol8w(T (&a)[4], int n, T tol, uint32_t mask, T* rbuf, T* diag0,
                                           int32_t* status) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int s = 0; s < 4; ++s)
    if (warp + 8 * s == lane) diag0[lane] = a[s];
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    T* rb = rbuf + (k & 1) * kSmallN;
    if (warp == (k & 7)) {
      const T ak = row_reg(a, k >> 3);
      const T d = __shfl_sync(0xffffffffu, ak, k);
      const T d0 = diag0[k];
      bool ok = (mask >> k) & 1u;
      if (!isfinite(d)) {
        ok = false;
        if (lane == 0) set_status(status, kStatusNotSpd);
      }
      if (!(d > tol * d0) || !(d0 > T(0))) ok = false;
      if (!ok && ((mask >> k) & 1u) && isfinite(d) && d0 > T(0) && lane == 0) note_dropped(status, k);
      const T yk = ok ? rsqrt_pivot(d) : T(0);
      const T rk = lane >= k ? ak * yk : T(0);
      set_row_reg(a, k >> 3, rk);
      rb[lane] = rk;
    }
    __syncthreads();
    const T rkc = rb[lane];
    if (!(rb[k] != T(0))) mask &= ~(1u << k);
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int i = warp + 8 * s;
      if (i > k && i < n && lane >= i) a[s] = fma(-rb[i], rkc, a[s]);
    }
  }
#pragma unroll
  for (int s = 0; s < 4; ++s)
    if (warp + 8 * s > lane) a[s] = T(0);
  return mask;
}

// W = R^{-1} on the same layout (R in a, upper triangular), backward and
// column-oriented: when row k of W is final (posted by warp k mod 8), every
// thread takes R[i][k] W[k][lane] off its rows i < k.  Rows and columns of
// dependent columns are zero.
template <typename T>
__device__ __forceinline__ void inv8w(const T (&a)[4], T (&w)[4], int n, uint32_t mask, T* wbuf, T* dinv) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int i = warp + 8 * s;
    if (i == lane && i < n) dinv[i] = ((mask >> i) & 1u) ? T(1) / a[s] : T(0);
    w[s] = i == lane ? T(1) : T(0);
  }
  __syncthreads();
  for (int k = n - 1; k >= 0; --k) {
    T* wb = wbuf + (k & 1) * kSmallN;
    if (warp == (k & 7)) {
      const T wk = row_reg(w, k >> 3) * dinv[k];
      set_row_reg(w, k >> 3, wk);
      wb[lane] = wk;
    }
    T rik[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) rik[s] = __shfl_sync(0xffffffffu, a[s], k);
    __syncthreads();
    const T wkc = wb[lane];
#pragma unroll
    for (int s = 0; s < 4; ++s)
      if (warp + 8 * s < k) w[s] = fma(-rik[s], wkc, w[s]);
  }
  if (!((mask >> lane) & 1u))
#pragma unroll
    for (int s = 0; s < 4; ++s) w[s] = T(0);
}

// First factorisation for n <= 32: R1 = chol(G1 + shift), W = R1^{-1} (8
// warps; the shift and from_r as in chol_first_body).
template <typename T>
__device__ __forceinline__ void chol_first32_body(const double* G, int n, double tol, double* R1, double* W, float* Wf,
                                                  int32_t* active, int32_t* status, double shift_rel, int from_r) {
  __shared__ T buf[2 * kSmallN], diag0[kSmallN], dinv[kSmallN];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool col = lane < n;
  const double shift = from_r ? 0.0 : gram_shift(G, n, shift_rel);
  T a[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int i = warp + 8 * s;
    const double g = (i < n && col) ? G[i * n + lane] : 0.0;
    a[s] = static_cast<T>(i == lane && g > 0.0 ? g + shift : g);
  }
  const uint32_t all = n >= 32 ? 0xffffffffu : ((1u << n) - 1u);
  const uint32_t mask =
      from_r ? __ballot_sync(0xffffffffu, col && G[lane * n + lane] != 0.0) & all
             : chol8w<T>(a, n, static_cast<T>(tol), all, buf, diag0, status);
  if (warp == 0 && col) active[lane] = (mask >> lane) & 1u;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int i = warp + 8 * s;
    if (i < n && col) R1[i * n + lane] = from_r ? (i <= lane && ((mask >> i) & 1u) ? G[i * n + lane] : 0.0)
                                                : static_cast<double>(a[s]);
  }
  __syncthreads();  // buf is reused by the inverse
  T w[4];
  inv8w<T>(a, w, n, mask, buf, dinv);
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int i = warp + 8 * s;
    if (i < n && col) {
      // dependent columns pass through the second pass unchanged (identity block)
      double v = i == lane && !((mask >> i) & 1u) ? 1.0 : static_cast<double>(w[s]);
      if (sizeof(T) == 4) {  // the value both Gram engines use exactly: hi (TF32) + lo rounded to TF32
        const float f = static_cast<float>(v);
        const float h = __uint_as_float(__float_as_uint(f) & 0xFFFFE000u);
        const float l = __uint_as_float((__float_as_uint(f - h) + 0x1000u) & 0xFFFFE000u);
        v = static_cast<double>(h + l);
      }
      W[i * n + lane] = v;
      Wf[i * n + lane] = static_cast<float>(v);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kC8Threads) chol_first32_kernel(const double* G, int n, double tol, double* R1,
                                                                  double* W, float* Wf, int32_t* active,
                                                                  int32_t* status, double shift_rel, int from_r) {
  pdl_enter();
  chol_first32_body<T>(G, n, tol, R1, W, Wf, active, status, shift_rel, from_r);
}

// Float-float helpers for the mixed path's second factorisation (FP64
// arithmetic is slow on this GPU): exact products by FMA, compensated sums.
__device__ __forceinline__ void ff_add_prod(float& hi, float& lo, float x, float y) {
  const float p = x * y;
  const float e = fmaf(x, y, -p);
  float s, t;
  two_sum(hi, p, s, t);
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(t, e));
}

// Second factorisation and R for n <= 32 (8 warps).  R2 = chol(G2) on the
// columns the first factorisation kept.  Mixed path (T = float): X = R1 + R1 E
// with E = I - W R1 formed in float-float from the exact FP32 values of W
// and R1, kept as the pair (R1, R1 E); R = R2 X in float-float.  Plain path
// (T = double): X = R1, R = R2 X in FP64.
template <typename T>
__device__ __forceinline__ void chol_second32_body(const double* G2, int n, double tol, const double* R1,
                                                   const float* Wf, const int32_t* active, int refine, double* R,
                                                   double* R_out, int64_t ldr, int32_t* status) {
  constexpr int LD = kSmallN + 1;
  __shared__ T buf[2 * kSmallN], diag0[kSmallN];
  __shared__ T sR2[kSmallN * LD], sX[kSmallN * LD];
  __shared__ float sW[kSmallN * LD], sE[kSmallN * LD], sXlo[kSmallN * LD];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool col = lane < n;
  const uint32_t mask1 = __ballot_sync(0xffffffffu, col && active[lane] != 0);
  T a[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int i = warp + 8 * s;
    a[s] = (i < n && col) ? static_cast<T>(G2[i * n + lane]) : T(0);
    // X = R1 on the independent columns, identity on the dependent diagonal
    T x = T(0);
    if (i < n && col && ((mask1 >> i) & 1u) && ((mask1 >> lane) & 1u)) x = static_cast<T>(R1[i * n + lane]);
    if (i == lane && col && !((mask1 >> i) & 1u)) x = T(1);
    sX[i * LD + lane] = x;
    if (refine) sW[i * LD + lane] = (i < n && col) ? Wf[i * n + lane] : 0.f;
  }
  const uint32_t mask2 = chol8w<T>(a, n, static_cast<T>(tol), mask1, buf, diag0, status);
  if (threadIdx.x == 0) header_of(status)->dep_cols = n - __popc(mask2 & (n >= 32 ? 0xffffffffu : ((1u << n) - 1u)));
#pragma unroll
  for (int s = 0; s < 4; ++s) sR2[(warp + 8 * s) * LD + lane] = a[s];
  if constexpr (sizeof(T) == 4) {
    if (refine) {
      // E = I - W R1 (upper triangle, independent columns), float-float
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int i = warp + 8 * s, j = lane;
        float e = 0.f;
        if (i <= j && j < n && ((mask1 >> i) & 1u) && ((mask1 >> j) & 1u)) {
          float hi = 0.f, lo = 0.f;
          for (int k = i; k <= j; ++k) ff_add_prod(hi, lo, sW[i * LD + k], sX[k * LD + j]);
          float t0, t1;
          two_sum(i == j ? 1.f : 0.f, -hi, t0, t1);
          e = __fadd_rn(t0, __fadd_rn(t1, -lo));
        }
        sE[i * LD + j] = e;
      }
      __syncthreads();
      // X = R1 + R1 E: the correction in FP32 (it is ~1e-7 of R1)
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int i = warp + 8 * s, j = lane;
        float c = 0.f;
        if (i <= j && j < n && ((mask1 >> i) & 1u) && ((mask1 >> j) & 1u))
          for (int k = i; k <= j; ++k) c = fmaf(sX[i * LD + k], sE[k * LD + j], c);
        sXlo[i * LD + j] = c;
      }
    } else {
#pragma unroll
      for (int s = 0; s < 4; ++s) sXlo[(warp + 8 * s) * LD + lane] = 0.f;
    }
  }
  __syncthreads();
  // R = R2 X (both upper triangular); rows of dependent columns are zero
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int i = warp + 8 * s, j = lane;
    if (i < n && j < n) {
      double r = 0.0;
      if (i <= j && sR2[i * LD + i] != T(0)) {
        if constexpr (sizeof(T) == 4) {
          float hi = 0.f, lo = 0.f;
          for (int k = i; k <= j; ++k) {
            const float r2 = sR2[i * LD + k];
            ff_add_prod(hi, lo, r2, sX[k * LD + j]);
            lo = fmaf(r2, sXlo[k * LD + j], lo);
          }
          r = static_cast<double>(hi) + static_cast<double>(lo);
        } else {
          double s0 = 0.0, s1 = 0.0;
          int k = i;
          for (; k + 1 <= j; k += 2) {
            s0 = fma(sR2[i * LD + k], sX[k * LD + j], s0);
            s1 = fma(sR2[i * LD + k + 1], sX[(k + 1) * LD + j], s1);
          }
          if (k <= j) s0 = fma(sR2[i * LD + k], sX[k * LD + j], s0);
          r = s0 + s1;
        }
      }
      R[i * n + j] = r;
      if (R_out) R_out[static_cast<int64_t>(i) * ldr + j] = r;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kC8Threads) chol_second32_kernel(const double* G2, int n, double tol,
                                                                   const double* R1, const float* Wf,
                                                                   const int32_t* active, int refine, double* R,
                                                                   double* R_out, int64_t ldr, int32_t* status) {
  pdl_enter();
  chol_second32_body<T>(G2, n, tol, R1, Wf, active, refine, R, R_out, ldr, status);
}

// One-sided Jacobi for n <= 32 with U (and V) in registers: lane l of each
// of the JW warps holds column l, warp w rows [RPW w, RPW (w + 1)), RPW =
// 32 / JW.  Rounds follow the circle method over np columns: column np - 1
// stays and the others rotate, so in round r lane l meets r if l = np - 1,
// np - 1 if l = r, and (2r - l) mod (np - 1) otherwise.  The two lanes of a
// pair swap their rows by shuffles and both form the partial 2 x 2 Gram of
// the lower-indexed column (x) against the higher one (y); the lower lane
// posts it, and after the round's barrier both sum the JW partials in warp
// order -- the same sums, hence the same rotation, in both lanes.  The
// convergence test, the negligible-column rule and the singular values
// (FP64 Rayleigh quotients with V, column norms without) are those of
// jacobi_body.
template <typename T, bool kWithV, int JW>
__device__ __forceinline__ void jacobi32_body(const double* R, int64_t ldr, int n, int max_sweeps, double tol_in,
                                              double* sigma, int32_t* status, int32_t* sweeps_out) {
  constexpr int RPW = kSmallN / JW;
  struct Part {
    T a, b, c, d;
  };
  __shared__ Part part[2][JW][kSmallN];
  __shared__ double red[JW][kSmallN];
  __shared__ double sig[kSmallN], unrm[kSmallN];
  __shared__ float Rh[kWithV ? kSmallN * kSmallN : 1], Rl[kWithV ? kSmallN * kSmallN : 1];  // R = Rh + Rl
  __shared__ T Vs[kWithV ? kSmallN * (kSmallN + 1) : 1];
  __shared__ float2 redf[JW][kSmallN];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int np = n + (n & 1), m = np - 1;
  T u[RPW], v[RPW];
#pragma unroll
  for (int t = 0; t < RPW; ++t) {
    const int row = warp * RPW + t;
    u[t] = (row < n && lane < n) ? static_cast<T>(R[static_cast<int64_t>(row) * ldr + lane]) : T(0);
    v[t] = (kWithV && row == lane && lane < n) ? T(1) : T(0);
  }
  if (kWithV)
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int i = e / n, k = e - i * n;
      const double r = R[static_cast<int64_t>(i) * ldr + k];
      const float h = static_cast<float>(r);
      Rh[i * kSmallN + k] = h;
      Rl[i * kSmallN + k] = static_cast<float>(r - static_cast<double>(h));
    }
  for (int e = threadIdx.x; e < 2 * JW * kSmallN; e += blockDim.x)
    (&part[0][0][0])[e] = Part{T(0), T(0), T(0), T(0)};  // idle lanes read slots nobody posts
  // ||R||_F^2 for the negligible-column rule
  {
    T f = T(0);
#pragma unroll
    for (int t = 0; t < RPW; ++t) f = fma(u[t], u[t], f);
    for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
    if (lane == 0) red[warp][0] = static_cast<double>(f);
  }
  __syncthreads();
  double fro = 0.0;
  for (int w = 0; w < JW; ++w) fro += red[w][0];
  const double eps64 = 1.1102230246251565e-16;
  const T negligible = static_cast<T>((n * eps64) * (n * eps64) * fro);
  const T tol2 = static_cast<T>(tol_in) * static_cast<T>(tol_in);
  __syncthreads();  // red[][0] is read above and written again below
  int sweep = 0, buf = 0;
  bool converged = false;
  for (; sweep < max_sweeps && !converged; ++sweep) {
    int any = 0;
    for (int r = 0; r < m; ++r) {
      int q = 2 * r - lane;  // (branch-free: the lanes of a warp take different cases)
      q += q < 0 ? m : 0;
      q -= q >= m ? m : 0;
      q = lane == r ? m : q;
      q = lane == m ? r : q;
      q = lane >= np ? lane : q;
      const bool lo = lane < q;
      // own and partner rows; the lower lane's (|own|^2, |other|^2, own.other)
      // over its rows is the pair's partial (alpha, beta, gamma)
      T o[RPW];
      T a = T(0), b = T(0), c = T(0);
#pragma unroll
      for (int t = 0; t < RPW; ++t) {
        o[t] = __shfl_sync(0xffffffffu, u[t], q);
        a = fma(u[t], u[t], a);
        b = fma(o[t], o[t], b);
        c = fma(u[t], o[t], c);
      }
      if (lo) part[buf][warp][lane] = Part{a, b, c, T(0)};
      __syncthreads();
      const int slot = lo ? lane : q;
      T al = T(0), be = T(0), ga = T(0);
#pragma unroll
      for (int w = 0; w < JW; ++w) {
        const Part p = part[buf][w][slot];
        al += p.a;
        be += p.b;
        ga += p.c;
      }
      buf ^= 1;
      const bool rot = q != lane && al > negligible && be > negligible && ga * ga > tol2 * al * be;
      // the rotation is formed in every lane (no divergent branch) and applied
      // as the identity where it is not wanted
      T cs, sn;
      rotation(al, be, rot ? ga : T(1), cs, sn);
      cs = rot ? cs : T(1);
      // lower column: c x - s y; upper column: s x + c y
      const T sg = rot ? (lo ? -sn : sn) : T(0);
#pragma unroll
      for (int t = 0; t < RPW; ++t) u[t] = fma(sg, o[t], cs * u[t]);
      if (kWithV) {
#pragma unroll
        for (int t = 0; t < RPW; ++t) {
          const T ov = __shfl_sync(0xffffffffu, v[t], q);
          v[t] = fma(sg, ov, cs * v[t]);
        }
      }
      any |= rot ? 1 : 0;
    }
    converged = __syncthreads_or(any) == 0;
  }
  if (!converged && threadIdx.x == 0) set_status(status, kStatusNoConvergence);
  if (threadIdx.x == 0 && sweeps_out) *sweeps_out = sweep;
  if (kWithV) {
    // Mixed path: the singular values are FP64-accurate Rayleigh quotients
    // sigma_j^2 = ||R v_j||^2 / ||v_j||^2, formed in float-float (R = Rh + Rl,
    // exact products by FMA; FP64 arithmetic is slow on this GPU) with one
    // FP64 division and square root per column.  Column norms ||u_j|| (the
    // fallback below 1e-3 sigma_max) likewise.
    {
      float uh = 0.f, ul = 0.f;
#pragma unroll
      for (int t = 0; t < RPW; ++t) ff_add_prod(uh, ul, static_cast<float>(u[t]), static_cast<float>(u[t]));
      redf[warp][lane] = make_float2(uh, ul);
#pragma unroll
      for (int t = 0; t < RPW; ++t) Vs[(warp * RPW + t) * (kSmallN + 1) + lane] = v[t];
    }
    __syncthreads();
    float2 un = make_float2(0.f, 0.f);
    if (warp == 0)
      for (int w = 0; w < JW; ++w) {
        float s_, e_;
        two_sum(un.x, redf[w][lane].x, s_, e_);
        un = make_float2(s_, __fadd_rn(un.y, __fadd_rn(e_, redf[w][lane].y)));
      }
    // thread (warp, lane): column j = lane, rows i = warp, warp + JW, ...
    const int j = lane;
    float nh = 0.f, nl = 0.f;
    if (j < n)
      for (int i = warp; i < n; i += JW) {
        float yh = 0.f, yl = 0.f;
        for (int k = i; k < n; ++k) {
          const float vk = static_cast<float>(Vs[k * (kSmallN + 1) + j]);
          ff_add_prod(yh, yl, Rh[i * kSmallN + k], vk);
          yl = fmaf(Rl[i * kSmallN + k], vk, yl);
        }
        float s_, e_;
        two_sum(yh, yl, s_, e_);  // normalise the pair before squaring
        ff_add_prod(nh, nl, s_, s_);
        nl = fmaf(2.f * s_, e_, nl);
      }
    __syncthreads();  // redf is read above by warp 0
    redf[warp][lane] = make_float2(nh, nl);
    __syncthreads();
    if (warp == 0) {
      float sh = 0.f, sl = 0.f, dh = 0.f, dl = 0.f;
      for (int w = 0; w < JW; ++w) {
        float s_, e_;
        two_sum(sh, redf[w][lane].x, s_, e_);
        sh = s_;
        sl = __fadd_rn(sl, __fadd_rn(e_, redf[w][lane].y));
      }
      for (int k = 0; k < n; ++k) {
        const float vk = static_cast<float>(Vs[k * (kSmallN + 1) + lane]);
        ff_add_prod(dh, dl, vk, vk);
      }
      const double unorm = sqrt(static_cast<double>(un.x) + static_cast<double>(un.y));
      unrm[lane] = lane < n ? unorm : 0.0;
      __syncwarp();
      double umax = 0.0;
      for (int k = 0; k < n; ++k) umax = unrm[k] > umax ? unrm[k] : umax;
      const double num = static_cast<double>(sh) + static_cast<double>(sl);
      const double den = static_cast<double>(dh) + static_cast<double>(dl);
      double sg = (lane < n && den > 0.0) ? sqrt(num / den) : 0.0;
      // below 1e-3 sigma_max the column norm is the more accurate value
      if (unorm < 1e-3 * umax) sg = unorm;
      sig[lane] = sg;
    }
  } else {
    // plain path: sigma_j = ||u_j|| in FP64
    double un = 0.0;
#pragma unroll
    for (int t = 0; t < RPW; ++t) un = fma(static_cast<double>(u[t]), static_cast<double>(u[t]), un);
    red[warp][lane] = un;
    __syncthreads();
    if (warp == 0) {
      double s_ = 0.0;
      for (int w = 0; w < JW; ++w) s_ += red[w][lane];
      sig[lane] = sqrt(s_);
    }
  }
  __syncthreads();
  if (threadIdx.x < n) {
    const int j = threadIdx.x;
    const double val = sig[j];
    int rank = 0;
    for (int k = 0; k < n; ++k) {
      const double w = sig[k];
      rank += (w > val) || (w == val && k < j);
    }
    sigma[rank] = val;
  }
}

template <typename T, bool kWithV, int JW>
__global__ void __launch_bounds__(32 * JW) jacobi32_kernel(const double* R, int64_t ldr, int n, int max_sweeps,
                                                           double tol_in, double* sigma, int32_t* status,
                                                           int32_t* sweeps_out) {
  pdl_enter();
  jacobi32_body<T, kWithV, JW>(R, ldr, n, max_sweeps, tol_in, sigma, status, sweeps_out);
}

// Warps of the register-resident Jacobi (rows per warp = 32 / JW).
constexpr int kJacobi32Warps = 4;

// ---- batched forms: one CTA per instance (job j = CTA j)
template <typename T, bool kSmall>
__global__ void __launch_bounds__(1024) chol_first_batched(BatchDev b, BatchJobs J) {
  pdl_enter();
  const Plan& P = b.plans[J.inst[blockIdx.x]];
  chol_first_body<T, kSmall>(P.G1, P.n, dense_tol(P), P.R1, P.W, P.Wf, P.active, &P.hdr->status, 0.0, 0);
}

template <typename T>
__global__ void __launch_bounds__(1024) chol_second_batched(BatchDev b, BatchJobs J) {
  pdl_enter();
  const int i = J.inst[blockIdx.x];
  const Plan& P = b.plans[i];
  if constexpr (sizeof(T) == 4) {
    if (P.mixed) {
      chol_second_ff_body(P.G2, P.n, dense_tol(P), P.R1, P.Wf, P.active, P.G1, P.R, b.out[i].R, P.n, &P.hdr->status);
      return;
    }
  }
  chol_second_body<T>(P.G2, P.n, dense_tol(P), P.R1, P.W, P.active, P.mixed, P.G1, P.R, b.out[i].R, P.n,
                      &P.hdr->status);
}

template <typename T, bool kWithV, int NPL>
__global__ void __launch_bounds__(512) jacobi_batched(BatchDev b, BatchJobs J) {
  pdl_enter();
  const int i = J.inst[blockIdx.x];
  const Plan& P = b.plans[i];
  jacobi_body<T, kWithV, NPL, kJacobiLPP>(P.R, P.n, P.n, P.max_sweeps, jacobi_tol(P), b.out[i].sigma, &P.hdr->status,
                                  &P.hdr->jacobi_sweeps);
}


template <typename T>
__global__ void __launch_bounds__(kC8Threads) chol_first32_batched(BatchDev b, BatchJobs J) {
  pdl_enter();
  const Plan& P = b.plans[J.inst[blockIdx.x]];
  chol_first32_body<T>(P.G1, P.n, dense_tol(P), P.R1, P.W, P.Wf, P.active, &P.hdr->status, 0.0, 0);
}

template <typename T>
__global__ void __launch_bounds__(kC8Threads) chol_second32_batched(BatchDev b, BatchJobs J) {
  pdl_enter();
  const int i = J.inst[blockIdx.x];
  const Plan& P = b.plans[i];
  chol_second32_body<T>(P.G2, P.n, dense_tol(P), P.R1, P.Wf, P.active, P.mixed, P.R, b.out[i].R, P.n,
                        &P.hdr->status);
}

template <typename T, bool kWithV>
__global__ void __launch_bounds__(32 * kJacobi32Warps) jacobi32_batched(BatchDev b, BatchJobs J) {
  pdl_enter();
  const int i = J.inst[blockIdx.x];
  const Plan& P = b.plans[i];
  jacobi32_body<T, kWithV, kJacobi32Warps>(P.R, P.n, P.n, P.max_sweeps, jacobi_tol(P), b.out[i].sigma,
                                           &P.hdr->status, &P.hdr->jacobi_sweeps);
}
}  // namespace

static double default_tol(const Plan& p) { return dense_tol(p); }

static int dense_threads(int n) {
  int t = 64;
  while (t < n * 32 && t < 1024) t <<= 1;
  return t;
}

// Relative shift of the shifted CholeskyQR3's first factorisation: 10 n u
// times trace(G1), u the unit roundoff of the Gram products (2^-24 on the
// mixed path, 2^-53 on the FP64 path).
static double shift_rel(const Plan& p) {
  if (!p.shifted) return 0.0;
  return 10.0 * p.n * (p.mixed ? 5.9604644775390625e-8 : 1.1102230246251565e-16);
}

template <typename T>
static cudaError_t chol_first_t(const Plan& p, cudaStream_t s, int from_r) {
  const int n = p.n;
  const double* G = from_r ? p.R : p.G1;
  const double sr = from_r ? 0.0 : shift_rel(p);
  // the column-per-thread inverse needs a second n x n buffer (when it fits)
  const bool small = sizeof(T) * 2 * static_cast<size_t>(n) * n <= 96 * 1024;
  size_t smem = sizeof(T) * (static_cast<size_t>(n) * n + 3 * n) + sizeof(int32_t) * (n + 4) + 16;
  if (small) smem += sizeof(T) * static_cast<size_t>(n) * n;
  if (n <= kSmallN) {
    pdl_launch(chol_first32_kernel<T>, 1, kC8Threads, 0, s, G, n, default_tol(p), p.R1, p.W, p.Wf, p.active,
               &p.hdr->status, sr, from_r);
    count_launches(1);
    return cudaGetLastError();
  }
  auto kern = small ? chol_first_kernel<T, true> : chol_first_kernel<T, false>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  pdl_launch(kern, 1, dense_threads(n), smem, s, G, n, default_tol(p), p.R1, p.W, p.Wf, p.active, &p.hdr->status,
             sr, from_r);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_chol_first(const Plan& p, cudaStream_t s) {
  if (p.wide) return launch_wide_chol_first(p, s);
  return p.mixed ? chol_first_t<float>(p, s, 0) : chol_first_t<double>(p, s, 0);
}

cudaError_t launch_refactor(const Plan& p, cudaStream_t s) {
  if (p.wide) return launch_wide_refactor(p, s);
  return p.mixed ? chol_first_t<float>(p, s, 1) : chol_first_t<double>(p, s, 1);
}

template <typename T>
static cudaError_t chol_second_t(const Plan& p, double* R_out, int64_t ldr, cudaStream_t s) {
  const int n = p.n;
  const size_t smem = chol_second_smem(n, p.mixed != 0);
  if (n <= kSmallN) {
    pdl_launch(chol_second32_kernel<T>, 1, kC8Threads, 0, s, p.G2, n, default_tol(p), p.R1, p.Wf, p.active,
               p.mixed ? 1 : 0, p.R, R_out, ldr, &p.hdr->status);
    count_launches(1);
    return cudaGetLastError();
  }
  auto kern = chol_second_kernel<T, false>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  // G1 is consumed by the first factorisation: its storage holds the refined inverse
  pdl_launch(kern, 1, dense_threads(n), smem, s, p.G2, n, default_tol(p), p.R1, p.W, p.Wf, p.active, p.mixed ? 1 : 0,
             p.G1, p.R, R_out, ldr, &p.hdr->status);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_chol_second(const Plan& p, double* R_out, int64_t ldr, cudaStream_t s) {
  if (p.wide) return launch_wide_chol_second(p, R_out, ldr, s);
  return p.mixed ? chol_second_t<float>(p, R_out, ldr, s) : chol_second_t<double>(p, R_out, ldr, s);
}

template <typename T, bool kWithV, int NPL, int LPP = 32>
static cudaError_t jacobi_t(const Plan& p, const double* R, int64_t ldr, double* sigma, double tol, cudaStream_t s) {
  const int n = p.n;
  const int np = n + (n & 1);
  const int npairs = np / 2;
  int threads = 32 * ((npairs + 32 / LPP - 1) / (32 / LPP));
  if (threads > 512) threads = 512;  // (the launch bound; n <= 128 needs at most 16 warps)
  const size_t smem = jacobi_smem(n, static_cast<int>(sizeof(T)), kWithV);
  cudaError_t err = cudaFuncSetAttribute(jacobi_kernel<T, kWithV, NPL, LPP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  pdl_launch(jacobi_kernel<T, kWithV, NPL, LPP>, 1, threads, smem, s, R, ldr, n, p.max_sweeps, tol, sigma, &p.hdr->status,
                                                               &p.hdr->jacobi_sweeps);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T, bool kWithV>
static cudaError_t jacobi32_t(const Plan& p, const double* R, int64_t ldr, double* sigma, double tol, cudaStream_t s) {
  pdl_launch(jacobi32_kernel<T, kWithV, kJacobi32Warps>, 1, 32 * kJacobi32Warps, 0, s, R, ldr, p.n, p.max_sweeps, tol,
             sigma, &p.hdr->status, &p.hdr->jacobi_sweeps);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_jacobi(const Plan& p, const double* R, int64_t ldr, double* sigma, cudaStream_t s) {
  if (p.wide) return launch_wide_jacobi(p, R, ldr, sigma, s);
  const int n = p.n;
  if (p.mixed) {
    // FP32 sweeps stop at |u_p . u_q| <= 1e-5 ||u_p|| ||u_q||: the FP64
    // Rayleigh quotient then has a relative error of order 1e-10 / gap
    if (n <= kSmallN) return jacobi32_t<float, true>(p, R, ldr, sigma, 1e-5, s);
    if (n <= 64) return jacobi_t<float, true, 8, kJacobiLPP>(p, R, ldr, sigma, 1e-5, s);
    return jacobi_t<float, true, 16, kJacobiLPP>(p, R, ldr, sigma, 1e-5, s);
  }
  const double tol = 4.0 * n * 1.1102230246251565e-16;
  if (n <= kSmallN) return jacobi32_t<double, false>(p, R, ldr, sigma, tol, s);
  if (n <= 64) return jacobi_t<double, false, 8, kJacobiLPP>(p, R, ldr, sigma, tol, s);
  return jacobi_t<double, false, 16, kJacobiLPP>(p, R, ldr, sigma, tol, s);
}

// Batched dense steps.  step 1: first Cholesky (variant 0: column-per-thread
// inverse with a second n x n buffer, 1: in-place inverse, 2: n <= 32 in one
// warp); step 2: second Cholesky and R (variant 1: n <= 32); step 3: Jacobi
// (variant 0: n <= 32 in registers, 1 and 2: 8 and 16 rows per lane, 8 lanes per pair).
template <typename T>
static size_t chol_first_smem(int n, bool small) {
  size_t smem = sizeof(T) * (static_cast<size_t>(n) * n + 3 * n) + sizeof(int32_t) * (n + 4) + 16;
  if (small) smem += sizeof(T) * static_cast<size_t>(n) * n;
  return smem;
}

void dense_batch_info(const Plan& p, int step, int* variant, size_t* smem, int* threads) {
  const int n = p.n;
  const size_t es = p.mixed ? 4 : 8;
  if (step == 1) {
    if (n <= kSmallN) {
      *variant = 2;
      *smem = 0;
      *threads = kC8Threads;
      return;
    }
    const bool small = es * 2 * static_cast<size_t>(n) * n <= 96 * 1024;
    *variant = small ? 0 : 1;
    *smem = p.mixed ? chol_first_smem<float>(n, small) : chol_first_smem<double>(n, small);
    *threads = dense_threads(n);
  } else if (step == 2) {
    if (n <= kSmallN) {
      *variant = 1;
      *smem = 0;
      *threads = kC8Threads;
      return;
    }
    *variant = 0;
    *smem = chol_second_smem(n, p.mixed != 0);
    *threads = dense_threads(n);
  } else {
    const int np = n + (n & 1), npairs = np / 2;
    *variant = n <= 32 ? 0 : (n <= 64 ? 1 : 2);
    if (n <= 32) {  // register-resident form
      *threads = 32 * kJacobi32Warps;
      *smem = 0;
      return;
    }
    constexpr int kPairsPerWarp = 32 / kJacobiLPP;
    int t = 32 * ((npairs + kPairsPerWarp - 1) / kPairsPerWarp);
    *threads = t > 512 ? 512 : t;  // (the launch bound)
    *smem = jacobi_smem(n, static_cast<int>(es), p.mixed != 0);
  }
}

template <typename K>
static cudaError_t launch_bucket(K kern, const BatchDev& b, const BatchJobs& J, size_t smem, int threads,
                                 cudaStream_t s) {
  if (J.njobs == 0) return cudaSuccess;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  pdl_launch(kern, J.njobs, threads, smem, s, b, J);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_batch_dense(const BatchDev& b, int step, const BatchJobs jobs[3], const size_t smem[3],
                               const int threads[3], int mixed, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (step == 1) {
    if (mixed) {
      e = launch_bucket(chol_first_batched<float, true>, b, jobs[0], smem[0], threads[0], s);
      if (e == cudaSuccess) e = launch_bucket(chol_first_batched<float, false>, b, jobs[1], smem[1], threads[1], s);
      if (e == cudaSuccess) e = launch_bucket(chol_first32_batched<float>, b, jobs[2], smem[2], threads[2], s);
    } else {
      e = launch_bucket(chol_first_batched<double, true>, b, jobs[0], smem[0], threads[0], s);
      if (e == cudaSuccess) e = launch_bucket(chol_first_batched<double, false>, b, jobs[1], smem[1], threads[1], s);
      if (e == cudaSuccess) e = launch_bucket(chol_first32_batched<double>, b, jobs[2], smem[2], threads[2], s);
    }
  } else if (step == 2) {
    e = mixed ? launch_bucket(chol_second_batched<float>, b, jobs[0], smem[0], threads[0], s)
              : launch_bucket(chol_second_batched<double>, b, jobs[0], smem[0], threads[0], s);
    if (e == cudaSuccess)
      e = mixed ? launch_bucket(chol_second32_batched<float>, b, jobs[1], smem[1], threads[1], s)
                : launch_bucket(chol_second32_batched<double>, b, jobs[1], smem[1], threads[1], s);
  } else {
    if (mixed) {
      e = launch_bucket(jacobi32_batched<float, true>, b, jobs[0], smem[0], threads[0], s);
      if (e == cudaSuccess) e = launch_bucket(jacobi_batched<float, true, 8>, b, jobs[1], smem[1], threads[1], s);
      if (e == cudaSuccess) e = launch_bucket(jacobi_batched<float, true, 16>, b, jobs[2], smem[2], threads[2], s);
    } else {
      e = launch_bucket(jacobi32_batched<double, false>, b, jobs[0], smem[0], threads[0], s);
      if (e == cudaSuccess) e = launch_bucket(jacobi_batched<double, false, 8>, b, jobs[1], smem[1], threads[1], s);
      if (e == cudaSuccess) e = launch_bucket(jacobi_batched<double, false, 16>, b, jobs[2], smem[2], threads[2], s);
    }
  }
  return e;
}

// Least squares over the join (Section 1's applications: the closed-form
// solution of linear regression).  With J = [J_x | y] (the label y is J's last
// column) and R = [[R11, r], [0, rho]] its QR factor, beta = R11^{-1} r
// minimises ||J_x beta - y|| and |rho| is the residual norm.  One warp, back
// substitution in FP64 (R staged in shared memory up to n = 128); a dependent
// feature column (zero row of R) gets beta_i = 0.
namespace {
constexpr int kLsqThreads = 256;

// R is staged in shared memory when it fits (n <= 128); beta lives there too.
__global__ void __launch_bounds__(kLsqThreads) lsq_kernel(const double* R, int n, double* beta, double* residual,
                                                          const int32_t* status, int staged) {
  pdl_enter();
  extern __shared__ __align__(16) double lsq_sm[];
  __shared__ double sb[kMaxWideWidth];
  if (*reinterpret_cast<const volatile int32_t*>(status) & kStatusTimeout) return;
  const int f = n - 1;  // features
  if (staged)
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) lsq_sm[e] = R[e];
  __syncthreads();
  const double* Rs = staged ? lsq_sm : R;
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int i = f - 1; i >= 0; --i) {
      const double* Ri = Rs + static_cast<int64_t>(i) * n;
      double s = 0.0;
      for (int k = i + 1 + lane; k < f; k += 32) s += Ri[k] * sb[k];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) sb[i] = Ri[i] != 0.0 ? (Ri[f] - s) / Ri[i] : 0.0;
      __syncwarp();
    }
    for (int i = lane; i < f; i += 32) beta[i] = sb[i];
    if (lane == 0) *residual = fabs(Rs[static_cast<int64_t>(f) * n + f]);
  }
}
}  // namespace

cudaError_t launch_lsq(const Plan& p, double* beta, double* residual, cudaStream_t s) {
  const int staged = p.n <= kMaxWidth ? 1 : 0;
  const size_t smem = staged ? sizeof(double) * static_cast<size_t>(p.n) * p.n : 0;
  cudaError_t err = cudaFuncSetAttribute(lsq_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  pdl_launch(lsq_kernel, 1, kLsqThreads, smem, s, static_cast<const double*>(p.R), p.n, beta, residual,
             static_cast<const int32_t*>(&p.hdr->status), staged);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace figaro
