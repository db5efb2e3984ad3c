// Small dense n x n steps of CholeskyQR2 and the singular values.  One CTA
// per instance (n <= 128), everything in shared memory.
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
// error of a few FP32 ulps -- while R = R2 R1 is formed in FP64; the Jacobi
// sweeps run in FP32 accumulating V and each singular value is then the FP64
// Rayleigh quotient ||R v_j|| / ||v_j||, whose error is second order in the
// FP32 error of v_j.  FP64 dependent chains are slow on this GPU (tens of
// cycles per FMA, hundreds per sqrt or divide), so the FP64 pivots use an
// FP32 seed refined by two Newton steps for 1/sqrt(d), and dot products are
// split across lanes.
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
    int ok = act[k];
    if (!isfinite(d)) ok = 0;
    if (!(d > tol * diag0[k]) || !(diag0[k] > T(0))) ok = 0;
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

template <typename T, bool kSmall>
__device__ __forceinline__ void chol_first_body(const double* G, int n, double tol, double* R1, double* W, float* Wf,
                                                int32_t* active, int32_t* status) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* A = reinterpret_cast<T*>(smraw);  // n x n
  T* diag0 = A + n * n;
  T* y = diag0 + n;
  T* x = y + n;
  int32_t* act = reinterpret_cast<int32_t*>(x + n);
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) A[e] = static_cast<T>(G[e]);
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    diag0[k] = static_cast<T>(G[k * n + k]);
    act[k] = 1;
  }
  __syncthreads();
  chol_inplace<T>(A, n, diag0, act, static_cast<T>(tol), y, status);
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    R1[e] = (j >= i && act[i]) ? static_cast<double>(A[e]) : 0.0;
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
                                  int32_t* active, int32_t* status) {
  pdl_enter();
  chol_first_body<T, kSmall>(G, n, tol, R1, W, Wf, active, status);
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
  // R = R2 X (both upper triangular) in FP64; rows of dependent columns are zero
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    const double s = (j >= i && act[i]) ? upper_dot(A, X, n, i, j) : 0.0;
    R[e] = s;
    if (R_out) R_out[static_cast<int64_t>(i) * ldr + j] = s;
  }
}

template <typename T, bool kSmall>
__global__ void __launch_bounds__(1024) chol_second_kernel(const double* G2, int n, double tol, const double* R1, const double* Wd,
                                   const int32_t* active, int refine, double* Xg, double* R, double* R_out,
                                   int64_t ldr, int32_t* status) {
  pdl_enter();
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

// One-sided Jacobi.  U (and V) column-major in shared memory; LPP lanes per
// column pair (32 / LPP pairs per warp), NPL rows of each column per lane;
// the round-robin pairing is tabulated once.  A pair is rotated while
// |u_p.u_q|^2 > tol^2 |u_p|^2 |u_q|^2.
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
          const int r = sub + LPP * i;
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
            const int r = sub + LPP * i;
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
              const int r = sub + LPP * i;
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
    // sigma_j^2 = sum_i (R v_j)_i^2 / ||v_j||^2 in FP64, one thread per (i, j).
    // U is no longer needed: its storage (np * n floats = np * n / 2 doubles)
    // holds the squared terms for np / 2 rows i at a time.
    double* acc = reinterpret_cast<double*>(U);
    for (int j = warp; j < n; j += nwarps) sig[j] = 0.0;
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
__global__ void __launch_bounds__(1024) jacobi_kernel(const double* R, int64_t ldr, int n, int max_sweeps, double tol_in, double* sigma,
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

// ---- batched forms: one CTA per instance (job j = CTA j)
template <typename T, bool kSmall>
__global__ void __launch_bounds__(1024) chol_first_batched(BatchDev b, BatchJobs J) {
  pdl_enter();
  const Plan& P = b.plans[J.inst[blockIdx.x]];
  chol_first_body<T, kSmall>(P.G1, P.n, dense_tol(P), P.R1, P.W, P.Wf, P.active, &P.hdr->status);
}

template <typename T>
__global__ void __launch_bounds__(1024) chol_second_batched(BatchDev b, BatchJobs J) {
  pdl_enter();
  const int i = J.inst[blockIdx.x];
  const Plan& P = b.plans[i];
  chol_second_body<T>(P.G2, P.n, dense_tol(P), P.R1, P.W, P.active, P.mixed, P.G1, P.R, b.out[i].R, P.n,
                      &P.hdr->status);
}

template <typename T, bool kWithV, int NPL>
__global__ void __launch_bounds__(1024) jacobi_batched(BatchDev b, BatchJobs J) {
  pdl_enter();
  const int i = J.inst[blockIdx.x];
  const Plan& P = b.plans[i];
  jacobi_body<T, kWithV, NPL, 32>(P.R, P.n, P.n, P.max_sweeps, jacobi_tol(P), b.out[i].sigma, &P.hdr->status,
                                  &P.hdr->jacobi_sweeps);
}

}  // namespace

static double default_tol(const Plan& p) { return dense_tol(p); }

static int dense_threads(int n) {
  int t = 64;
  while (t < n * 32 && t < 1024) t <<= 1;
  return t;
}

template <typename T>
static cudaError_t chol_first_t(const Plan& p, cudaStream_t s) {
  const int n = p.n;
  // the column-per-thread inverse needs a second n x n buffer (when it fits)
  const bool small = sizeof(T) * 2 * static_cast<size_t>(n) * n <= 96 * 1024;
  size_t smem = sizeof(T) * (static_cast<size_t>(n) * n + 3 * n) + sizeof(int32_t) * (n + 4) + 16;
  if (small) smem += sizeof(T) * static_cast<size_t>(n) * n;
  auto kern = small ? chol_first_kernel<T, true> : chol_first_kernel<T, false>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  pdl_launch(kern, 1, dense_threads(n), smem, s, p.G1, n, default_tol(p), p.R1, p.W, p.Wf, p.active, &p.hdr->status);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_chol_first(const Plan& p, cudaStream_t s) {
  if (p.wide) return launch_wide_chol_first(p, s);
  return p.mixed ? chol_first_t<float>(p, s) : chol_first_t<double>(p, s);
}

template <typename T>
static cudaError_t chol_second_t(const Plan& p, double* R_out, int64_t ldr, cudaStream_t s) {
  const int n = p.n;
  size_t smem = ((sizeof(T) * (static_cast<size_t>(n) * n + 2 * n) + sizeof(int32_t) * n + 15) & ~size_t(15));
  if (p.mixed) smem += sizeof(double) * static_cast<size_t>(n) * n;
  auto kern = chol_second_kernel<T, false>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  // G1 is consumed by the first factorisation: its storage holds the refined inverse
  pdl_launch(kern, 1, dense_threads(n), smem, s, p.G2, n, default_tol(p), p.R1, p.W, p.active, p.mixed ? 1 : 0, p.G1, p.R,
                                         R_out, ldr, &p.hdr->status);
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
  if (threads > 1024) threads = 1024;
  size_t smem = sizeof(T) * static_cast<size_t>(np) * n * (kWithV ? 2 : 1) + 2 * sizeof(double) * np;
  if (kWithV && n <= 64) smem += sizeof(double) * static_cast<size_t>(n) * n;
  smem += sizeof(short2) * static_cast<size_t>(np - 1) * npairs;
  cudaError_t err = cudaFuncSetAttribute(jacobi_kernel<T, kWithV, NPL, LPP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  pdl_launch(jacobi_kernel<T, kWithV, NPL, LPP>, 1, threads, smem, s, R, ldr, n, p.max_sweeps, tol, sigma, &p.hdr->status,
                                                               &p.hdr->jacobi_sweeps);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_jacobi(const Plan& p, const double* R, int64_t ldr, double* sigma, cudaStream_t s) {
  if (p.wide) return launch_wide_jacobi(p, R, ldr, sigma, s);
  const int n = p.n;
  if (p.mixed) {
    // FP32 sweeps stop at |u_p . u_q| <= 1e-5 ||u_p|| ||u_q||: the FP64
    // Rayleigh quotient then has a relative error of order 1e-10 / gap
    if (n <= 32) return jacobi_t<float, true, 1>(p, R, ldr, sigma, 1e-5, s);
    if (n <= 64) return jacobi_t<float, true, 2>(p, R, ldr, sigma, 1e-5, s);
    return jacobi_t<float, true, 4>(p, R, ldr, sigma, 1e-5, s);
  }
  const double tol = 4.0 * n * 1.1102230246251565e-16;
  if (n <= 32) return jacobi_t<double, false, 1>(p, R, ldr, sigma, tol, s);
  if (n <= 64) return jacobi_t<double, false, 2>(p, R, ldr, sigma, tol, s);
  return jacobi_t<double, false, 4>(p, R, ldr, sigma, tol, s);
}

// Batched dense steps.  step 1: first Cholesky (variant 0: column-per-thread
// inverse with a second n x n buffer, 1: in-place inverse); step 2: second
// Cholesky and R; step 3: Jacobi (variant = rows per lane 1, 2, 4 -> 0, 1, 2).
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
    const bool small = es * 2 * static_cast<size_t>(n) * n <= 96 * 1024;
    *variant = small ? 0 : 1;
    *smem = p.mixed ? chol_first_smem<float>(n, small) : chol_first_smem<double>(n, small);
    *threads = dense_threads(n);
  } else if (step == 2) {
    *variant = 0;
    *smem = ((es * (static_cast<size_t>(n) * n + 2 * n) + sizeof(int32_t) * n + 15) & ~size_t(15)) +
            (p.mixed ? sizeof(double) * static_cast<size_t>(n) * n : 0);
    *threads = dense_threads(n);
  } else {
    const int np = n + (n & 1), npairs = np / 2;
    const int npl = n <= 32 ? 1 : (n <= 64 ? 2 : 4);
    *variant = npl == 1 ? 0 : (npl == 2 ? 1 : 2);
    int t = 32 * npairs;  // one warp per pair (32 lanes per pair)
    *threads = t > 1024 ? 1024 : t;
    const bool with_v = p.mixed != 0;
    size_t sm = es * static_cast<size_t>(np) * n * (with_v ? 2 : 1) + 2 * sizeof(double) * np;
    if (with_v && n <= 64) sm += sizeof(double) * static_cast<size_t>(n) * n;
    sm += sizeof(short2) * static_cast<size_t>(np - 1) * npairs;
    *smem = sm;
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
    } else {
      e = launch_bucket(chol_first_batched<double, true>, b, jobs[0], smem[0], threads[0], s);
      if (e == cudaSuccess) e = launch_bucket(chol_first_batched<double, false>, b, jobs[1], smem[1], threads[1], s);
    }
  } else if (step == 2) {
    e = mixed ? launch_bucket(chol_second_batched<float>, b, jobs[0], smem[0], threads[0], s)
              : launch_bucket(chol_second_batched<double>, b, jobs[0], smem[0], threads[0], s);
  } else {
    if (mixed) {
      e = launch_bucket(jacobi_batched<float, true, 1>, b, jobs[0], smem[0], threads[0], s);
      if (e == cudaSuccess) e = launch_bucket(jacobi_batched<float, true, 2>, b, jobs[1], smem[1], threads[1], s);
      if (e == cudaSuccess) e = launch_bucket(jacobi_batched<float, true, 4>, b, jobs[2], smem[2], threads[2], s);
    } else {
      e = launch_bucket(jacobi_batched<double, false, 1>, b, jobs[0], smem[0], threads[0], s);
      if (e == cudaSuccess) e = launch_bucket(jacobi_batched<double, false, 2>, b, jobs[1], smem[1], threads[1], s);
      if (e == cudaSuccess) e = launch_bucket(jacobi_batched<double, false, 4>, b, jobs[2], smem[2], threads[2], s);
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
