// Small dense n x n steps of CholeskyQR2 and the singular values.
//
//  * chol_first:  R1 = chol(G1) (FP64, semi-definite: a pivot below
//                 rank_tol * G1_kk marks column k as dependent and gives a
//                 zero row), W = R1^{-1} on the independent columns.
//  * chol_second: R2 = chol(G2) on the same columns, R = R2 R1 (FP64); the
//                 diagonal is positive, so R already has the sign convention
//                 of Section 1 (R is the Cholesky factor of J^T J).
//  * jacobi:      one-sided (Hestenes) Jacobi on the columns of R (Section 3:
//                 the singular values of J are those of R), parallel
//                 round-robin ordering, one thread group per column pair.
//                 Plain path: FP64 sweeps, sigma = column norms.  Mixed
//                 path: FP32 sweeps accumulating V, then sigma_j =
//                 ||R v_j|| / ||v_j|| in FP64 (a Rayleigh quotient, so the
//                 FP32 error of v_j enters only to second order).
// All three run as one CTA per instance (n <= 128).
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace figaro {
namespace {

// In-place semi-definite Cholesky of the n x n matrix A (shared memory,
// row-major, upper triangle used).  act[k] (in/out): columns marked 0 on
// entry stay dependent.  Returns via A the upper factor with zero rows for
// dependent columns.
__device__ void chol_inplace(double* A, int n, const double* diag0, int32_t* act, double tol, int32_t* status) {
  __shared__ double s_inv;
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      double d = A[k * n + k];
      int ok = act[k];
      if (!isfinite(d)) {
        set_status(status, kStatusNotSpd);
        ok = 0;
      }
      if (!(d > tol * diag0[k]) || !(diag0[k] > 0.0)) ok = 0;
      act[k] = ok;
      if (ok) {
        double r = sqrt(d);
        A[k * n + k] = r;
        s_inv = 1.0 / r;
      } else {
        A[k * n + k] = 0.0;
        s_inv = 0.0;
      }
    }
    __syncthreads();
    const double inv = s_inv;
    for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) A[k * n + j] *= inv;
    __syncthreads();
    if (inv != 0.0) {
      const int m = n - k - 1;  // trailing (i, j) with k < i <= j < n
      for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        int a = e / m, b = e - a * m;
        if (b < a) continue;
        int i = k + 1 + a, j = k + 1 + b;
        A[i * n + j] -= A[k * n + i] * A[k * n + j];
      }
    }
    __syncthreads();
  }
}

__global__ void chol_first_kernel(const double* G, int n, double tol, double* R1, double* W, float* Wf,
                                  int32_t* active, int32_t* status) {
  extern __shared__ double sm[];
  double* A = sm;                // n x n
  double* diag0 = sm + n * n;    // n
  int32_t* act = reinterpret_cast<int32_t*>(diag0 + n);
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) A[e] = G[e];
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    diag0[k] = G[k * n + k];
    act[k] = 1;
  }
  __syncthreads();
  chol_inplace(A, n, diag0, act, tol, status);
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int i = e / n, j = e % n;
    R1[e] = (j >= i && act[i]) ? A[e] : 0.0;
  }
  for (int k = threadIdx.x; k < n; k += blockDim.x) active[k] = act[k];
  __syncthreads();
  // W = R1^{-1} on the independent columns, in place (column j of W needs
  // only W's leading j x j block and column j of R1).
  double* x = diag0;  // reuse as a length-n temporary
  for (int j = 0; j < n; ++j) {
    const bool aj = act[j] != 0;
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
      double s = 0.0;
      if (aj && act[i])
        for (int k = i; k < j; ++k) s += A[i * n + k] * A[k * n + j];
      x[i] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) A[j * n + j] = aj ? 1.0 / A[j * n + j] : 0.0;
    __syncthreads();
    const double wjj = A[j * n + j];
    for (int i = threadIdx.x; i < j; i += blockDim.x) A[i * n + j] = (aj && act[i]) ? -x[i] * wjj : 0.0;
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int i = e / n, j = e % n;
    double w = (j >= i) ? A[e] : 0.0;
    W[e] = w;
    Wf[e] = static_cast<float>(w);
  }
}

__global__ void chol_second_kernel(const double* G2, int n, double tol, const double* R1, const int32_t* active,
                                   double* R, double* R_out, int64_t ldr, int32_t* status) {
  extern __shared__ double sm[];
  double* A = sm;
  double* diag0 = sm + n * n;
  int32_t* act = reinterpret_cast<int32_t*>(diag0 + n);
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) A[e] = G2[e];
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    diag0[k] = G2[k * n + k];
    act[k] = active[k];
  }
  __syncthreads();
  chol_inplace(A, n, diag0, act, tol, status);
  // R = R2 R1 (both upper triangular); rows of dependent columns are zero
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int i = e / n, j = e % n;
    double s = 0.0;
    if (j >= i && act[i]) {
      for (int k = i; k <= j; ++k) s += A[i * n + k] * R1[k * n + j];
    }
    R[e] = s;
    if (R_out) R_out[static_cast<int64_t>(i) * ldr + j] = s;
  }
}

template <typename T>
__device__ __forceinline__ T group_sum(T v, int width) {
  for (int o = width >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, width);
  return v;
}

// One-sided Jacobi.  U (and V) column-major in shared memory.
template <typename T, bool kWithV>
__global__ void jacobi_kernel(const double* R, int64_t ldr, int n, int max_sweeps, int tpp, double* sigma,
                              int32_t* status, int32_t* sweeps_out) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int np = n + (n & 1);  // even number of columns (one zero column if n is odd)
  T* U = reinterpret_cast<T*>(smraw);
  T* V = U + static_cast<int64_t>(np) * n;
  double* sig = reinterpret_cast<double*>(smraw + sizeof(T) * static_cast<size_t>(np) * n * (kWithV ? 2 : 1));
  __shared__ int s_rot;
  for (int e = threadIdx.x; e < np * n; e += blockDim.x) {
    int c = e / n, r = e % n;
    U[e] = c < n ? static_cast<T>(R[static_cast<int64_t>(r) * ldr + c]) : T(0);
    if (kWithV) V[e] = (c == r) ? T(1) : T(0);
  }
  __syncthreads();
  // rotate while |u_p . u_q| > tol ||u_p|| ||u_q||; 4 n eps leaves room for the rounding of the dot products
  const T eps = sizeof(T) == 4 ? T(5.9604645e-8) : T(1.1102230246251565e-16);
  const T tol = T(4) * static_cast<T>(n) * eps;
  // columns whose squared norm is below (n eps)^2 ||R||_F^2 are rounding
  // noise of a rank-deficient R: they take no part in rotations
  __shared__ T s_fro;
  if (threadIdx.x < 32) {
    T f = 0;
    for (int e = threadIdx.x; e < np * n; e += 32) f += U[e] * U[e];
    for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
    if (threadIdx.x == 0) s_fro = f;
  }
  __syncthreads();
  const T negligible = (static_cast<T>(n) * eps) * (static_cast<T>(n) * eps) * s_fro;
  const int group = threadIdx.x / tpp;
  const int gl = threadIdx.x % tpp;
  const int npairs = np / 2;
  int sweep = 0;
  bool converged = false;
  __syncthreads();
  for (; sweep < max_sweeps && !converged; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int round = 0; round < np - 1; ++round) {
      {
        const bool real = group < npairs;
        int p, q;
        if (!real) {
          p = 0;
          q = 1;
        } else if (group == 0) {
          p = round;
          q = np - 1;
        } else {
          p = (round + group) % (np - 1);
          q = (round - group + (np - 1)) % (np - 1);
        }
        if (p > q) {
          int t = p;
          p = q;
          q = t;
        }
        T* up = U + static_cast<int64_t>(p) * n;
        T* uq = U + static_cast<int64_t>(q) * n;
        T al = 0, be = 0, ga = 0;
        for (int r = gl; r < n; r += tpp) {
          T x = up[r], y = uq[r];
          al += x * x;
          be += y * y;
          ga += x * y;
        }
        al = group_sum(al, tpp);
        be = group_sum(be, tpp);
        ga = group_sum(ga, tpp);
        bool rotate = real && al > negligible && be > negligible && ga != T(0) && fabs(ga) > tol * sqrt(al * be);
        if (rotate) {
          T zeta = (be - al) / (T(2) * ga);
          T t = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
          T c = T(1) / sqrt(T(1) + t * t);
          T s = c * t;
          for (int r = gl; r < n; r += tpp) {
            T x = up[r], y = uq[r];
            up[r] = c * x - s * y;
            uq[r] = s * x + c * y;
          }
          if (kWithV) {
            T* vp = V + static_cast<int64_t>(p) * n;
            T* vq = V + static_cast<int64_t>(q) * n;
            for (int r = gl; r < n; r += tpp) {
              T x = vp[r], y = vq[r];
              vp[r] = c * x - s * y;
              vq[r] = s * x + c * y;
            }
          }
          if (gl == 0) s_rot = 1;
        }
      }
      __syncthreads();
    }
    converged = s_rot == 0;
    __syncthreads();
  }
  if (!converged) {
    if (threadIdx.x == 0) set_status(status, kStatusNoConvergence);
  }
  if (threadIdx.x == 0 && sweeps_out) *sweeps_out = sweep;
  // singular values
  const int warps = blockDim.x / 32, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int j = wid; j < n; j += warps) {
    double num = 0.0, den = 0.0;
    if (kWithV) {
      const T* vj = V + static_cast<int64_t>(j) * n;
      for (int i = lane; i < n; i += 32) {
        double y = 0.0;
        for (int k = i; k < n; ++k) y += R[static_cast<int64_t>(i) * ldr + k] * static_cast<double>(vj[k]);
        num += y * y;
        double v = static_cast<double>(vj[i]);
        den += v * v;
      }
    } else {
      const T* uj = U + static_cast<int64_t>(j) * n;
      for (int i = lane; i < n; i += 32) {
        double u = static_cast<double>(uj[i]);
        num += u * u;
      }
      den = 1.0;
    }
    for (int o = 16; o > 0; o >>= 1) {
      num += __shfl_xor_sync(0xffffffffu, num, o);
      if (kWithV) den += __shfl_xor_sync(0xffffffffu, den, o);
    }
    if (lane == 0) sig[j] = den > 0.0 ? sqrt(num / den) : 0.0;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double v = sig[j];
    int rank = 0;
    for (int k = 0; k < n; ++k) {
      double w = sig[k];
      rank += (w > v) || (w == v && k < j);
    }
    sigma[rank] = v;
  }
}

}  // namespace

static double default_tol(const Plan& p) { return p.rank_tol > 0 ? p.rank_tol : (p.mixed ? 1e-5 : 1e-13); }

static int dense_threads(int n) {
  int t = 32;
  while (t < n * 8 && t < 1024) t <<= 1;
  return t;
}

cudaError_t launch_chol_first(const Plan& p, cudaStream_t s) {
  int n = p.n;
  size_t smem = sizeof(double) * (static_cast<size_t>(n) * n + n) + sizeof(int32_t) * n;
  cudaError_t err = cudaFuncSetAttribute(chol_first_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  chol_first_kernel<<<1, dense_threads(n), smem, s>>>(p.G1, n, default_tol(p), p.R1, p.W, p.Wf, p.active,
                                                        &p.hdr->status);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_chol_second(const Plan& p, double* R_out, int64_t ldr, cudaStream_t s) {
  int n = p.n;
  size_t smem = sizeof(double) * (static_cast<size_t>(n) * n + n) + sizeof(int32_t) * n;
  cudaError_t err = cudaFuncSetAttribute(chol_second_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  chol_second_kernel<<<1, dense_threads(n), smem, s>>>(p.G2, n, default_tol(p), p.R1, p.active, p.R, R_out, ldr,
                                                         &p.hdr->status);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_jacobi(const Plan& p, const double* R, int64_t ldr, double* sigma, cudaStream_t s) {
  int n = p.n;
  int np = n + (n & 1);
  int pairs = np / 2;
  int tpp = 32;
  while (tpp > 1 && tpp * pairs > 1024) tpp >>= 1;
  int threads = tpp * pairs;
  if (threads < 32) threads = 32;
  threads = (threads + 31) / 32 * 32;
  cudaError_t err;
  if (p.mixed) {
    size_t smem = sizeof(float) * static_cast<size_t>(np) * n * 2 + sizeof(double) * n;
    err = cudaFuncSetAttribute(jacobi_kernel<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    jacobi_kernel<float, true><<<1, threads, smem, s>>>(R, ldr, n, p.max_sweeps, tpp, sigma, &p.hdr->status,
                                                         &p.hdr->jacobi_sweeps);
  } else {
    size_t smem = sizeof(double) * static_cast<size_t>(np) * n + sizeof(double) * n;
    err = cudaFuncSetAttribute(jacobi_kernel<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    jacobi_kernel<double, false><<<1, threads, smem, s>>>(R, ldr, n, p.max_sweeps, tpp, sigma, &p.hdr->status,
                                                           &p.hdr->jacobi_sweeps);
  }
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace figaro
