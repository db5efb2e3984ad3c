// Device helpers shared by the Figaro kernels (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace figaro {

// Device status bits, recorded in the workspace header; the host maps them
// to figaro_status (the lowest set bit's code wins).
enum : int32_t {
  kStatusNotSpd = 1 << 4,
  kStatusNoConvergence = 1 << 5,
  kStatusTimeout = 1 << 6,
  // a factorisation marked a column with a non-zero norm dependent (its pivot
  // fell below rank_tol times its diagonal) and the call reports that column
  kStatusRankDrop = 1 << 7,
  // FIGARO_FLAG_PRESORTED was set but a table's keys are not in ascending order
  kStatusUnsorted = 1 << 8,
};

__device__ __forceinline__ void set_status(int32_t* word, int32_t bit) { atomicOr(word, bit); }

// Programmatic dependent launch: every kernel first waits until the kernel
// before it in the stream has completed and its memory is visible, then lets
// the next kernel be scheduled while it runs (both are no-ops for a launch
// without the programmatic-serialization attribute).
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Keys: int32 mapped to uint32 so that unsigned order equals signed order.
__device__ __forceinline__ uint32_t key_to_ordered(int32_t k) { return static_cast<uint32_t>(k) ^ 0x80000000u; }
__device__ __forceinline__ int32_t ordered_to_key(uint32_t u) { return static_cast<int32_t>(u ^ 0x80000000u); }

// Acquire / release accesses for the cross-CTA look-back protocol.
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Error-free transformation of a + b (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// 1/sqrt(d) for d > 0: FP32 estimate refined by Newton's iteration
// y <- y (3 - d y^2) / 2 (quadratic convergence; two steps from ~2^-23).
__device__ __forceinline__ double rsqrt_pivot(double d) {
  if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
  double y = static_cast<double>(rsqrtf(static_cast<float>(d)));
  y = y * (1.5 - 0.5 * d * y * y);
  y = y * (1.5 - 0.5 * d * y * y);
  return y;
}
__device__ __forceinline__ float rsqrt_pivot(float d) { return __frsqrt_rn(d); }

// Compensated accumulator: float-float pair for FP32, plain sum for FP64.
template <typename T>
struct Acc;

template <>
struct Acc<float> {
  float hi, lo;
  __device__ __forceinline__ void zero() { hi = 0.f; lo = 0.f; }
  __device__ __forceinline__ void add(float x) {
    float s, e;
    two_sum(hi, x, s, e);
    hi = s;
    lo = __fadd_rn(lo, e);
  }
  __device__ __forceinline__ void add(const Acc<float>& o) {
    float s, e;
    two_sum(hi, o.hi, s, e);
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(e, o.lo));
  }
  __device__ __forceinline__ void set_double(double d) {
    hi = static_cast<float>(d);
    lo = static_cast<float>(d - static_cast<double>(hi));
  }
  __device__ __forceinline__ double to_double() const { return static_cast<double>(hi) + static_cast<double>(lo); }
  __device__ __forceinline__ float value() const { return __fadd_rn(hi, lo); }
};

template <>
struct Acc<double> {
  double v;
  __device__ __forceinline__ void zero() { v = 0.0; }
  __device__ __forceinline__ void add(double x) { v += x; }
  __device__ __forceinline__ void add(const Acc<double>& o) { v += o.v; }
  __device__ __forceinline__ void set_double(double d) { v = d; }
  __device__ __forceinline__ double to_double() const { return v; }
  __device__ __forceinline__ double value() const { return v; }
};

template <typename T>
__device__ __forceinline__ Acc<T> shfl_up_acc(const Acc<T>& a, int delta);

template <>
__device__ __forceinline__ Acc<float> shfl_up_acc(const Acc<float>& a, int delta) {
  Acc<float> r;
  r.hi = __shfl_up_sync(0xffffffffu, a.hi, delta);
  r.lo = __shfl_up_sync(0xffffffffu, a.lo, delta);
  return r;
}
template <>
__device__ __forceinline__ Acc<double> shfl_up_acc(const Acc<double>& a, int delta) {
  Acc<double> r;
  r.v = __shfl_up_sync(0xffffffffu, a.v, delta);
  return r;
}

}  // namespace figaro
