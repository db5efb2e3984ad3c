// Gram products of the reduced matrix on 5th-generation tensor cores
// (tcgen05, kind::tf32), the mixed-precision engine of the CholeskyQR2
// passes (same block structure and meaning as gram.cu).
//
// Precision: every FP32 operand v is split as v = hi + lo with hi = v with
// its 13 low mantissa bits cleared (exactly TF32) and lo = v - hi rounded to
// TF32; a product is formed from hi*hi + hi*lo + lo*hi (3xTF32), so each term
// carries ~22 significant bits.  For the symmetric Gram the two correction
// terms are one MMA: with lo' = 2 lo the block accumulates P = H + 2 C
// (H = hi^T hi, C = hi^T lo) and the reduction takes G = (P + P^T) / 2 =
// H + C + C^T exactly.  The tensor core rounds its FP32 accumulator toward
// zero at every MMA, a bias that grows with the number of MMAs adding large
// values into one accumulator; so a 128-row tile goes to four accumulators
// of 32 rows each (small correction terms first, the large hi*hi terms
// last), drained after every tile (summed in FP32 with round-to-nearest)
// into float-float accumulators held in registers; the block's partial is
// written in FP64 at the end (partials are reduced in a fixed order).
//
// Per block (128 threads; thread t owns row t of a 128-row tile):
//   1. TMA loads the next X tile (128 rows x k in 32-column panels) one tile
//      ahead (two buffers, mbarrier transaction counts).  Pass 1 loads it with
//      the 32-byte-atom 128-byte swizzle, the layout the tensor core reads
//      TF32 operands from when M or N (here: the columns of X) is the
//      contiguous dimension; pass 2 with the plain 128-byte swizzle, the
//      K-major layout of the formation product.
//   2. The tile is split elementwise: hi in place, lo into a second buffer.
//   3. Pass 2 only: three formation MMAs D1 = X W (M = 128 rows, N = kout,
//      K = k) into tensor memory; each thread reads its row of D1 back
//      (tcgen05.ld), splits it and writes the hi / lo rows of Q contiguously
//      in the 32-byte-atom layout.
//   4. Gram MMAs hi^T lo' and hi^T hi (Q = X in pass 1; M = 64 or 128,
//      N = kout, K = 128 rows, both operands MN-major) into the four
//      accumulators; the previous tile's accumulators are drained first.
// A single elected thread issues every MMA and TMA; completion is tracked
// with tcgen05.commit -> mbarrier.  Every wait is bounded: on timeout the
// block records FIGARO_ERR_DEVICE_TIMEOUT, stops issuing work, waits (again
// bounded) for what it issued, frees its tensor memory and exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace figaro {
namespace {

constexpr int kTcThreads = 128;
constexpr int kTileRows = 128;
constexpr int kPanelBytes = kTileRows * 128;  // one 32-column panel of an X tile
constexpr int kHiAcc = 4;  // accumulators per tile of the pipelined engine (4 K-steps of 8 rows each)
constexpr int kTcAcc = 2;  // accumulators per tile of the general engine (8 K-steps each; with the formation
                           // buffer 3 x 64 columns of tensor memory, so that two CTAs share an SM)

struct TcArgs {
  int k;             // columns of X (multiple of 4)
  int kout;          // Gram width
  int kpanels;       // ceil(k / 32): 128-byte panels of an X row
  int ksteps_f;      // formation K steps of 8 (k padded to 8)
  int np;            // kout padded to 16 (N of both MMAs)
  int mg;            // Gram M: 64 or 128
  int qpanels;       // ceil(kout / 32): 32-column panels of a Q row
  int wpanel_bytes;  // np * 128
  int64_t rows;
  const int64_t* rows_dev;
  const float* W;    // pass 2: W block base (row-major, leading dimension wld); nullptr for pass 1
  int wld;
  double* part;      // [grid][kout][kout]
  int32_t* status;
  int64_t spin_limit;
  // shared memory offsets (bytes from the 1024-aligned base)
  int off_x[2], off_xlo, off_wh, off_wl, off_qh, off_ql;
  int alias;         // pass 2, wide Q: one X buffer, Q's lo part over X and its lo part (two CTAs per SM)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor, K-major, 128-byte swizzle (layout type 2):
// 8-row groups 1,024 bytes apart.
__device__ __forceinline__ uint64_t desc_kmajor_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFF);
  d |= static_cast<uint64_t>(1) << 16;                    // leading byte offset (unused for swizzled K-major)
  d |= static_cast<uint64_t>(1024 >> 4) << 32;            // stride byte offset
  d |= static_cast<uint64_t>(1) << 46;                    // descriptor version
  d |= static_cast<uint64_t>(2) << 61;                    // 128-byte swizzle
  return d;
}

// Shared-memory matrix descriptor, MN-major TF32 in the 128-byte swizzle with
// 32-byte atoms (layout type 1): 4-row groups 512 bytes apart, 32-column
// panels `panel` bytes apart (0 repeats the first panel).
__device__ __forceinline__ uint64_t desc_mn_sw128_32b(uint32_t saddr, uint32_t panel) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFF);
  d |= static_cast<uint64_t>((panel >> 4) & 0x3FFF) << 16;  // leading byte offset: next 32 M/N columns
  d |= static_cast<uint64_t>(512 >> 4) << 32;              // stride byte offset: next 4 K rows
  d |= static_cast<uint64_t>(1) << 46;
  d |= static_cast<uint64_t>(1) << 61;
  return d;
}

// Instruction descriptor: kind::tf32, FP32 accumulator; mn = 1 makes both
// operands MN-major (A = M x K with M contiguous, B = K x N with N contiguous).
__device__ __forceinline__ uint32_t idesc_tf32(int M, int N, int mn = 0) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(mn) << 15) | (static_cast<uint32_t>(mn) << 16) |
         (static_cast<uint32_t>(N >> 3) << 17) | (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p; }" ::"r"(dtmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

// One lane of the (converged) warp, chosen by the hardware.
__device__ __forceinline__ bool elect_one() {
  uint32_t e;
  asm volatile("{ .reg .pred p; elect.sync _|p, 0xffffffff; selp.u32 %0, 1, 0, p; }" : "=r"(e));
  return e != 0;
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* b, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}

// Bounded wait for the given phase parity; false if the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, int64_t limit) {
  for (int64_t i = 0; i < limit; ++i) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// L2 prefetch of the same box (no shared memory, no completion to track).
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap* map, int x, int y) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(map), "r"(x), "r"(y) : "memory");
}

__device__ __forceinline__ void expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ float tf32_hi(float v) { return __uint_as_float(__float_as_uint(v) & 0xFFFFE000u); }
// Round to the nearest TF32 value, ties away from zero (the tie rule does not
// enter the error bounds of the splits).
__device__ __forceinline__ float tf32_rn(float v) {
  return __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xFFFFE000u);
}

// 32 consecutive TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* out) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int c = 0; c < 32; ++c) out[c] = __uint_as_float(r[c]);
}

// Byte offset of element (row, col) of a 128-byte-swizzled K-major panel set:
// 32 columns per panel, rows of 128 bytes, 16-byte chunks XOR (row mod 8).
__device__ __forceinline__ int sw128_offset(int row, int col, int panel_bytes) {
  const int p = col >> 5, kk = col & 31;
  return p * panel_bytes + row * 128 + ((((kk >> 2) ^ (row & 7))) << 4) + ((kk & 3) << 2);
}

// Byte offset of the 32-byte chunk holding columns [8c, 8c + 8) of a row in
// the 32-byte-atom 128-byte swizzle: chunk c of row r sits at chunk c ^ (r mod 4).
__device__ __forceinline__ int sw32b_chunk_offset(int row, int chunk) {
  return ((chunk >> 2) * kTileRows * 128) + row * 128 + (((chunk & 3) ^ (row & 3)) << 5);
}

template <int NP>
__device__ __forceinline__ void gram_tc_body(const CUtensorMap* tmx, const TcArgs& a, int cta, int G) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t bar_tma[2], bar_f, bar_g;
  __shared__ uint32_t tmem_base;
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5;
  const bool pass2 = a.W != nullptr;
  const int64_t rows = a.rows_dev ? *a.rows_dev : a.rows;
  const int64_t ntiles = (rows + kTileRows - 1) / kTileRows;
  // formation result + kTcAcc Gram accumulators, NP columns each
  constexpr uint32_t kCols = (kTcAcc + 1) * NP;
  const uint32_t tmem_cols = kCols <= 32 ? 32 : (kCols <= 64 ? 64 : (kCols <= 128 ? 128 : (kCols <= 256 ? 256 : 512)));

  if (tid == 0) {
    mbar_init(&bar_tma[0], 1);
    mbar_init(&bar_tma[1], 1);
    mbar_init(&bar_f, 1);
    mbar_init(&bar_g, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (pass2) {  // W^T (np rows x k, K-major): hi and lo parts; padding rows / columns are zero
    float* wh = reinterpret_cast<float*>(base + a.off_wh);
    float* wl = reinterpret_cast<float*>(base + a.off_wl);
    const int wbytes = a.kpanels * a.wpanel_bytes;
    for (int e = tid; e < wbytes / 4; e += kTcThreads) {
      wh[e] = 0.f;
      wl[e] = 0.f;
    }
    __syncthreads();
    for (int e = tid; e < a.kout * a.k; e += kTcThreads) {
      const int n = e / a.k, kk = e - n * a.k;
      const float v = (kk <= n) ? a.W[static_cast<int64_t>(kk) * a.wld + n] : 0.f;  // W upper triangular
      const int off = sw128_offset(n, kk, a.wpanel_bytes);
      const float h = tf32_hi(v);
      *reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(wh) + off) = h;
      *reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(wl) + off) = tf32_rn(v - h);
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t d1 = tmem;                                   // formation result: 128 lanes x NP
  const uint32_t dacc = tmem + static_cast<uint32_t>(NP);    // kTcAcc Gram accumulators of NP columns
  const uint32_t tile_bytes = static_cast<uint32_t>(a.kpanels * kPanelBytes);

  // prologue: the first tile of this block (each later tile is loaded one
  // iteration ahead, into the buffer the previous tile's MMAs released)
  if (tid == 0 && static_cast<int64_t>(cta) < ntiles) {
    expect_tx(&bar_tma[0], tile_bytes);
    for (int p = 0; p < a.kpanels; ++p)
      tma_load_2d(base + a.off_x[0] + p * kPanelBytes, tmx, p * 32, static_cast<int>(cta * kTileRows),
                  &bar_tma[0]);
  }

  // Gram row held by this thread's TMEM lane (M = 64: 16 rows per 32-lane quarter)
  const int lane_row = a.mg == 64 ? (((tid & 31) < 16) ? (warp * 16 + (tid & 31)) : -1) : tid;
  float acc_hi[NP], acc_lo[NP];  // float-float running sums of that row
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    acc_hi[j] = 0.f;
    acc_lo[j] = 0.f;
  }
  // drain the accumulators of the tile whose Gram MMAs just completed
  auto drain = [&]() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
    for (int c0 = 0; c0 < NP; c0 += 32) {
      float sum[32], v[32];
      tmem_ld32(dacc + (static_cast<uint32_t>(warp * 32) << 16) + c0, sum);
#pragma unroll 1
      for (int q = 1; q < kTcAcc; ++q) {
        tmem_ld32(dacc + (static_cast<uint32_t>(warp * 32) << 16) + q * NP + c0, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) sum[j] = __fadd_rn(sum[j], v[j]);
      }
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        float s_, e_;
        two_sum(acc_hi[c0 + j], sum[j], s_, e_);
        acc_hi[c0 + j] = s_;
        acc_lo[c0 + j] = __fadd_rn(acc_lo[c0 + j], e_);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  };

  const uint32_t panel_mn = a.kpanels > 1 || a.qpanels > 1 ? static_cast<uint32_t>(kPanelBytes) : 0u;
  int it = 0;
  bool pending_g = false;  // Gram MMAs committed and not yet waited for
  uint32_t g_phase = 0, f_phase = 0;
  for (int64_t rt = cta; rt < ntiles; rt += G, ++it) {
    const int buf = a.alias ? 0 : (it & 1);
    float* X = reinterpret_cast<float*>(base + a.off_x[buf]);
    float* Xl = reinterpret_cast<float*>(base + a.off_xlo);
    if (pending_g) {  // the previous tile's Gram MMAs: operands and accumulators become free
      if (!mbar_wait(&bar_g, g_phase, a.spin_limit)) {
        if (tid == 0) {
          set_status(a.status, kStatusTimeout);
          s_abort = 1;
        }
      }
      g_phase ^= 1;
      pending_g = false;
      __syncthreads();
      if (s_abort) break;
      drain();
    }
    if (tid == 0) {
      if (!a.alias) {  // the other buffer is free: load the next tile into it
        const int64_t nt = rt + static_cast<int64_t>(G);
        if (nt < ntiles) {
          expect_tx(&bar_tma[buf ^ 1], tile_bytes);
          for (int p = 0; p < a.kpanels; ++p)
            tma_load_2d(base + a.off_x[buf ^ 1] + p * kPanelBytes, tmx, p * 32, static_cast<int>(nt * kTileRows),
                        &bar_tma[buf ^ 1]);
        }
      } else if (it > 0) {  // one buffer (the first tile came with the prologue): the previous Gram is done
        expect_tx(&bar_tma[0], tile_bytes);
        for (int p = 0; p < a.kpanels; ++p)
          tma_load_2d(base + a.off_x[0] + p * kPanelBytes, tmx, p * 32, static_cast<int>(rt * kTileRows), &bar_tma[0]);
      }
    }
    if (!mbar_wait(&bar_tma[buf], static_cast<uint32_t>(a.alias ? (it & 1) : ((it >> 1) & 1)), a.spin_limit)) {
      if (tid == 0) {
        set_status(a.status, kStatusTimeout);
        s_abort = 1;
      }
    }
    __syncthreads();
    if (s_abort) break;
    // split X elementwise: hi in place, lo in the second buffer (same layout;
    // 2 lo when it feeds the Gram, lo when it feeds the formation product);
    // rows past the end (head block: count known on the device) are zeroed
    {
      const float lo_scale = pass2 ? 1.f : 2.f;
      float4* X4 = reinterpret_cast<float4*>(X);
      float4* L4 = reinterpret_cast<float4*>(Xl);
      const int n4 = static_cast<int>(tile_bytes / 16);
      for (int e = tid; e < n4; e += kTcThreads) {
        const int row = (e % (kTileRows * 8)) / 8;  // 8 float4 per 128-byte row, panels of kTileRows rows
        float4 v = X4[e];
        if (rt * kTileRows + row >= rows) v = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 h, l;
        h.x = tf32_hi(v.x); h.y = tf32_hi(v.y); h.z = tf32_hi(v.z); h.w = tf32_hi(v.w);
        l.x = tf32_rn(v.x - h.x) * lo_scale; l.y = tf32_rn(v.y - h.y) * lo_scale;
        l.z = tf32_rn(v.z - h.z) * lo_scale; l.w = tf32_rn(v.w - h.w) * lo_scale;
        X4[e] = h;
        L4[e] = l;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    uint32_t ah = smem_u32(X), al = smem_u32(Xl);
    if (pass2) {
      if (warp == 0) {  // D1 = X W (3 x TF32), the large term last
        // the warp runs the issue (descriptors built once: their address
        // field is bytes / 16, so K steps are constants added to a base),
        // one elected lane issues the straight run of MMAs
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const bool leader = elect_one();
        const uint32_t idf = idesc_tf32(128, a.np);
        const uint64_t dah = desc_kmajor_sw128(ah), dal = desc_kmajor_sw128(al);
        const uint64_t dwh = desc_kmajor_sw128(smem_u32(base + a.off_wh));
        const uint64_t dwl = desc_kmajor_sw128(smem_u32(base + a.off_wl));
        const int wp16 = a.wpanel_bytes >> 4, ksf = a.ksteps_f;
        if (leader) {
#pragma unroll
          for (int ks = 0; ks < 8; ++ks)
            if (ks < ksf) {
              const uint64_t ao = static_cast<uint64_t>((ks >> 2) * (kPanelBytes >> 4) + (ks & 3) * 2);
              const uint64_t bo = static_cast<uint64_t>((ks >> 2) * wp16 + (ks & 3) * 2);
              mma_tf32(d1, dal + ao, dwh + bo, idf, ks > 0 ? 1u : 0u);
              mma_tf32(d1, dah + ao, dwl + bo, idf, 1u);
            }
#pragma unroll
          for (int ks = 0; ks < 8; ++ks)
            if (ks < ksf) {
              const uint64_t ao = static_cast<uint64_t>((ks >> 2) * (kPanelBytes >> 4) + (ks & 3) * 2);
              const uint64_t bo = static_cast<uint64_t>((ks >> 2) * wp16 + (ks & 3) * 2);
              mma_tf32(d1, dah + ao, dwh + bo, idf, 1u);
            }
          mma_commit(&bar_f);
        }
        __syncwarp();
      }
      if (!mbar_wait(&bar_f, f_phase, a.spin_limit)) {
        if (tid == 0) {
          set_status(a.status, kStatusTimeout);
          s_abort = 1;
        }
      }
      f_phase ^= 1;
      __syncthreads();
      if (s_abort) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // row tid of Q = X W: split and write contiguously (32-byte-atom layout)
      unsigned char* qh = base + a.off_qh;
      unsigned char* ql = base + a.off_ql;
#pragma unroll
      for (int c0 = 0; c0 < NP; c0 += 32) {
        if (c0 >= a.qpanels * 32) break;
        float q[32];
        tmem_ld32(d1 + (static_cast<uint32_t>(warp * 32) << 16) + c0, q);
        if (rt * kTileRows + tid >= rows) {
#pragma unroll
          for (int c = 0; c < 32; ++c) q[c] = 0.f;
        }
#pragma unroll
        for (int ch = 0; ch < 4; ++ch) {
          const int off = sw32b_chunk_offset(tid, (c0 >> 3) + ch);
          float4 h0, h1, l0, l1;
          const float* v = q + ch * 8;
          h0 = make_float4(tf32_hi(v[0]), tf32_hi(v[1]), tf32_hi(v[2]), tf32_hi(v[3]));
          h1 = make_float4(tf32_hi(v[4]), tf32_hi(v[5]), tf32_hi(v[6]), tf32_hi(v[7]));
          l0 = make_float4(2.f * tf32_rn(v[0] - h0.x), 2.f * tf32_rn(v[1] - h0.y), 2.f * tf32_rn(v[2] - h0.z),
                           2.f * tf32_rn(v[3] - h0.w));
          l1 = make_float4(2.f * tf32_rn(v[4] - h1.x), 2.f * tf32_rn(v[5] - h1.y), 2.f * tf32_rn(v[6] - h1.z),
                           2.f * tf32_rn(v[7] - h1.w));
          reinterpret_cast<float4*>(qh + off)[0] = h0;
          reinterpret_cast<float4*>(qh + off)[1] = h1;
          reinterpret_cast<float4*>(ql + off)[0] = l0;
          reinterpret_cast<float4*>(ql + off)[1] = l1;
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      ah = smem_u32(qh);
      al = smem_u32(ql);
    }
    if (warp == 0) {  // Gram MMAs, both operands MN-major: P += hi^T (2 lo) + hi^T hi (issued as the formation)
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const bool leader = elect_one();
      const uint32_t idg = idesc_tf32(a.mg, a.np, 1);
      constexpr int kSteps = kTileRows / 8, kPer = kSteps / kTcAcc;
      const uint64_t dh = desc_mn_sw128_32b(ah, panel_mn), dl = desc_mn_sw128_32b(al, panel_mn);
      if (leader) {
#pragma unroll
        for (int q = 0; q < kTcAcc; ++q) {
          const uint32_t d = dacc + static_cast<uint32_t>(q * NP);
#pragma unroll
          for (int s = 0; s < kPer; ++s) {
            const uint64_t o = static_cast<uint64_t>(((q * kPer + s) * 1024) >> 4);
            mma_tf32(d, dh + o, dl + o, idg, s > 0 ? 1u : 0u);
          }
#pragma unroll
          for (int s = 0; s < kPer; ++s) {
            const uint64_t o = static_cast<uint64_t>(((q * kPer + s) * 1024) >> 4);
            mma_tf32(d, dh + o, dh + o, idg, 1u);
          }
        }
        mma_commit(&bar_g);
      }
      __syncwarp();
    }
    pending_g = true;
  }
  // the last tile's Gram MMAs, then their accumulators
  if (pending_g) {
    if (!mbar_wait(&bar_g, g_phase, a.spin_limit)) {
      if (tid == 0) set_status(a.status, kStatusTimeout);
      s_abort = 1;
    }
    __syncthreads();
    if (!s_abort) drain();
  }
  double* part = a.part + static_cast<int64_t>(cta) * a.kout * a.kout;
  if (lane_row >= 0 && lane_row < a.kout) {
#pragma unroll
    for (int j = 0; j < NP; ++j)
      if (j < a.kout) part[lane_row * a.kout + j] = static_cast<double>(acc_hi[j]) + static_cast<double>(acc_lo[j]);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
}

template <int NP>
__global__ void __launch_bounds__(kTcThreads) gram_tc_kernel(const __grid_constant__ CUtensorMap tmx, TcArgs a) {
  pdl_enter();
  gram_tc_body<NP>(&tmx, a, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// Pipelined engine for k <= 32 and kout <= 32 (one 32-column panel per row).
//
// Warp roles (10 warps):
//   warp 0     TMA producer: X tiles into a ring of kPipeStages stages.
//   warp 1     allocates tensor memory; one thread issues every MMA.
//   warps 2-9  workers: split each landed tile (hi in place, lo in the
//              stage's second buffer); pass 2: read the formation result
//              D1 = X W back from tensor memory (warp w reads TMEM lanes
//              32 (w mod 4) .. + 31, half of the columns each), split Q and
//              write it as the Gram operands; drain the Gram accumulators.
// Double buffers in tensor memory (D1 and the Gram accumulator sets) let
// the MMAs of tile i overlap the workers' draining of tile i - 1.  The
// workers sum the four accumulators of a tile in FP32 (round to nearest),
// add up to kDrainGroup tiles in FP32 and fold that into float-float sums.
// Every wait is bounded; a timeout sets the status bit and an abort flag
// that makes every role leave its loop.
constexpr int kPipeStages = 4;
constexpr int kWorkWarps = 8;
constexpr int kPipeThreads = 64 + 32 * kWorkWarps;
constexpr int kDrainGroup = 8;

struct PipeArgs {
  int k, kout, np, ksteps_f;
  int64_t rows;
  const int64_t* rows_dev;
  const float* W;  // pass 2: W block base (row-major, leading dimension wld); nullptr for pass 1
  int wld;
  double* part;    // [grid][kout][kout]
  int32_t* status;
  int64_t spin_limit;
};

struct PipeSmem {
  uint64_t tma_full[kPipeStages], stage_empty[kPipeStages], op_full[kPipeStages];
  uint64_t d1_full[2], d1_empty[2], q_full[2], q_empty[2], acc_full[2], acc_empty[2], done;
  uint32_t tmem_base;
  int abort;
};

// byte offsets from the 1024-aligned dynamic base
constexpr int kOffRaw = 0;                                   // kPipeStages x 16 KB
constexpr int kOffLo = kOffRaw + kPipeStages * kPanelBytes;  // kPipeStages x 16 KB
constexpr int kOffQh = kOffLo + kPipeStages * kPanelBytes;   // 2 x 16 KB
constexpr int kOffQl = kOffQh + 2 * kPanelBytes;             // 2 x 16 KB
constexpr int kOffWh = kOffQl + 2 * kPanelBytes;             // 32 rows x 128 B
constexpr int kOffWl = kOffWh + 32 * 128;
constexpr int kPipeSmemBytes = kOffWl + 32 * 128 + 1024;

// The waiting thread is suspended in hardware between tries (hint 1 us), so
// waiting warps do not take issue slots from the working ones.
__device__ __forceinline__ bool pipe_wait(PipeSmem& S, uint64_t* b, uint32_t parity, int64_t limit, int32_t* status) {
  const int64_t tries = limit / 16 + 1;
  for (int64_t i = 0; i < tries; ++i) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity), "r"(1000u)
        : "memory");
    if (ok) return true;
    if (*reinterpret_cast<volatile int*>(&S.abort)) return false;
  }
  set_status(status, kStatusTimeout);
  *reinterpret_cast<volatile int*>(&S.abort) = 1;
  return false;
}

// Bounded wait that ignores the abort flag: used before the CTA exits, for
// copies and MMAs already issued.
__device__ __forceinline__ void drain_wait(uint64_t* b, uint32_t parity, int64_t limit, int32_t* status) {
  for (int64_t i = 0; i < limit; ++i) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    if (ok) return;
  }
  set_status(status, kStatusTimeout);
}

// A warp waits through its lane 0 (the other lanes do not poll); __syncwarp
// then orders what lane 0 observed before the rest of the warp reads it.
__device__ __forceinline__ bool warp_wait(PipeSmem& S, uint64_t* b, uint32_t parity, int64_t limit, int32_t* status) {
  int ok = 1;
  if ((threadIdx.x & 31) == 0) ok = pipe_wait(S, b, parity, limit, status) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  __syncwarp();
  return ok != 0;
}

// Non-blocking test of a phase parity.
__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

// One lane of the (fully active) warp: the issuer of a warp-wide MMA loop.
__device__ __forceinline__ void mbar_arrive_cta(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

// 16 consecutive TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* out) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int c = 0; c < 16; ++c) out[c] = __uint_as_float(r[c]);
}

__global__ void __launch_bounds__(kPipeThreads, 1)
    gram_pipe_kernel(const __grid_constant__ CUtensorMap tmx, PipeArgs a) {
  pdl_enter();
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ PipeSmem S;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool pass2 = a.W != nullptr;
  const int64_t rows = a.rows_dev ? *a.rows_dev : a.rows;
  const int64_t ntiles_all = (rows + kTileRows - 1) / kTileRows;
  const int G = gridDim.x;
  const int n = ntiles_all > blockIdx.x ? static_cast<int>((ntiles_all - 1 - blockIdx.x) / G + 1) : 0;
  auto tile_row0 = [&](int i) -> int64_t { return (static_cast<int64_t>(blockIdx.x) + static_cast<int64_t>(i) * G) * kTileRows; };

  if (tid == 0) {
    for (int q = 0; q < kPipeStages; ++q) {
      mbar_init(&S.tma_full[q], 1);
      mbar_init(&S.stage_empty[q], 1);
      mbar_init(&S.op_full[q], kWorkWarps);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&S.d1_full[b], 1);
      mbar_init(&S.d1_empty[b], kWorkWarps);
      mbar_init(&S.q_full[b], kWorkWarps);
      mbar_init(&S.q_empty[b], 1);
      mbar_init(&S.acc_full[b], 1);
      mbar_init(&S.acc_empty[b], kWorkWarps);
    }
    mbar_init(&S.done, 1);
    S.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (pass2 && warp >= 2) {  // W^T (np rows x k, K-major 128-byte swizzle): hi and lo parts, zero padded
    const int wt = tid - 64;
    float* wh = reinterpret_cast<float*>(base + kOffWh);
    float* wl = reinterpret_cast<float*>(base + kOffWl);
    for (int e = wt; e < 32 * 32; e += 32 * kWorkWarps) {
      wh[e] = 0.f;
      wl[e] = 0.f;
    }
    asm volatile("bar.sync 1, %0;" ::"n"(32 * kWorkWarps) : "memory");
    for (int e = wt; e < a.kout * a.k; e += 32 * kWorkWarps) {
      const int nn = e / a.k, kk = e - nn * a.k;
      const float v = (kk <= nn) ? a.W[static_cast<int64_t>(kk) * a.wld + nn] : 0.f;  // W upper triangular
      const int off = sw128_offset(nn, kk, 32 * 128);
      const float h = tf32_hi(v);
      *reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(wh) + off) = h;
      *reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(wl) + off) = tf32_rn(v - h);
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = S.tmem_base;
  auto d1_addr = [&](int b) { return tmem + static_cast<uint32_t>(b * 32); };
  auto acc_addr = [&](int b, int q) { return tmem + 64u + static_cast<uint32_t>(b * 128 + q * 32); };

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int issued = 0;
      for (int i = 0; i < n; ++i) {
        const int s = i % kPipeStages;
        if (i >= kPipeStages &&
            !pipe_wait(S, &S.stage_empty[s], static_cast<uint32_t>(((i / kPipeStages) - 1) & 1), a.spin_limit, a.status))
          break;
        expect_tx(&S.tma_full[s], kPanelBytes);
        tma_load_2d(base + kOffRaw + s * kPanelBytes, &tmx, 0, static_cast<int>(tile_row0(i)), &S.tma_full[s]);
        issued = i + 1;
      }
      // every load issued has landed before the CTA may exit (bounded)
      for (int i = issued > kPipeStages ? issued - kPipeStages : 0; i < issued; ++i)
        drain_wait(&S.tma_full[i % kPipeStages], static_cast<uint32_t>((i / kPipeStages) & 1), a.spin_limit, a.status);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      const uint32_t idg = idesc_tf32(64, a.np, 1);
      const uint32_t idf = idesc_tf32(128, a.np);
      const uint32_t wh = smem_u32(base + kOffWh), wl = smem_u32(base + kOffWl);
      // descriptors are linear in the start address (bits 0-13 hold addr >> 4),
      // so a K step of 8 rows (1,024 bytes) adds 64
      auto gram = [&](uint32_t ah, uint32_t al, int b) {
        constexpr int kSteps = kTileRows / 8, kPer = kSteps / kHiAcc;
        const uint64_t dh = desc_mn_sw128_32b(ah, 0), dl = desc_mn_sw128_32b(al, 0);
        // round robin over the independent accumulators (consecutive MMAs do
        // not depend on each other); per accumulator the small terms come first
#pragma unroll
        for (int st = 0; st < kPer; ++st)
#pragma unroll
          for (int q = 0; q < kHiAcc; ++q) {
            const uint64_t o = static_cast<uint64_t>((q * kPer + st) * 64);
            mma_tf32(acc_addr(b, q), dh + o, dl + o, idg, st > 0 ? 1u : 0u);
          }
#pragma unroll
        for (int st = 0; st < kPer; ++st)
#pragma unroll
          for (int q = 0; q < kHiAcc; ++q) {
            const uint64_t o = static_cast<uint64_t>((q * kPer + st) * 64);
            mma_tf32(acc_addr(b, q), dh + o, dh + o, idg, 1u);
          }
      };
      auto formation = [&](int j) -> bool {  // D1[j & 1] = X_j W (3 x TF32, the large term last)
        const int s = j % kPipeStages, bd = j & 1;
        if (!pipe_wait(S, &S.op_full[s], static_cast<uint32_t>((j / kPipeStages) & 1), a.spin_limit, a.status))
          return false;
        if (j >= 2 && !pipe_wait(S, &S.d1_empty[bd], static_cast<uint32_t>(((j / 2) - 1) & 1), a.spin_limit, a.status))
          return false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t ah = smem_u32(base + kOffRaw + s * kPanelBytes), al = smem_u32(base + kOffLo + s * kPanelBytes);
        for (int ks = 0; ks < a.ksteps_f; ++ks) {
          const uint32_t o = static_cast<uint32_t>(ks * 32);
          mma_tf32(d1_addr(bd), desc_kmajor_sw128(al + o), desc_kmajor_sw128(wh + o), idf, ks > 0 ? 1u : 0u);
          mma_tf32(d1_addr(bd), desc_kmajor_sw128(ah + o), desc_kmajor_sw128(wl + o), idf, 1u);
        }
        for (int ks = 0; ks < a.ksteps_f; ++ks) {
          const uint32_t o = static_cast<uint32_t>(ks * 32);
          mma_tf32(d1_addr(bd), desc_kmajor_sw128(ah + o), desc_kmajor_sw128(wh + o), idf, 1u);
        }
        mma_commit(&S.stage_empty[s]);
        mma_commit(&S.d1_full[bd]);
        return true;
      };
      if (!pass2) {
        for (int i = 0; i < n; ++i) {
          const int s = i % kPipeStages, b = i & 1;
          if (!pipe_wait(S, &S.op_full[s], static_cast<uint32_t>((i / kPipeStages) & 1), a.spin_limit, a.status)) break;
          if (i >= 2 && !pipe_wait(S, &S.acc_empty[b], static_cast<uint32_t>(((i / 2) - 1) & 1), a.spin_limit, a.status))
            break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          gram(smem_u32(base + kOffRaw + s * kPanelBytes), smem_u32(base + kOffLo + s * kPanelBytes), b);
          mma_commit(&S.stage_empty[s]);
          mma_commit(&S.acc_full[b]);
        }
      } else if (n > 0 && formation(0)) {
        for (int i = 0; i < n; ++i) {
          const int b = i & 1;
          if (i + 1 < n && !formation(i + 1)) break;
          if (!pipe_wait(S, &S.q_full[b], static_cast<uint32_t>((i / 2) & 1), a.spin_limit, a.status)) break;
          if (i >= 2 && !pipe_wait(S, &S.acc_empty[b], static_cast<uint32_t>(((i / 2) - 1) & 1), a.spin_limit, a.status))
            break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          gram(smem_u32(base + kOffQh + b * kPanelBytes), smem_u32(base + kOffQl + b * kPanelBytes), b);
          mma_commit(&S.q_empty[b]);
          mma_commit(&S.acc_full[b]);
        }
      }
      // all MMAs issued by this thread have completed before tensor memory is freed (bounded)
      mma_commit(&S.done);
      drain_wait(&S.done, 0u, a.spin_limit, a.status);
    }
  } else {
    // ------------------------------------------------------------ workers
    const int wt = tid - 64;
    const int quarter = warp & 3, half = (warp - 2) >> 2;
    const int c0 = half * 16;  // this warp's 16 columns of D1 and of the accumulators
    const float lo_scale = pass2 ? 1.f : 2.f;
    auto split = [&](int i) -> bool {
      const int s = i % kPipeStages;
      if (!pipe_wait(S, &S.tma_full[s], static_cast<uint32_t>((i / kPipeStages) & 1), a.spin_limit, a.status))
        return false;
      float4* X4 = reinterpret_cast<float4*>(base + kOffRaw + s * kPanelBytes);
      float4* L4 = reinterpret_cast<float4*>(base + kOffLo + s * kPanelBytes);
      const int64_t r0 = tile_row0(i);
      for (int e = wt; e < kPanelBytes / 16; e += 32 * kWorkWarps) {
        const int row = e >> 3;  // 8 float4 per 128-byte row
        float4 v = X4[e];
        if (r0 + row >= rows) v = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 h, l;
        h.x = tf32_hi(v.x); h.y = tf32_hi(v.y); h.z = tf32_hi(v.z); h.w = tf32_hi(v.w);
        l.x = tf32_rn(v.x - h.x) * lo_scale; l.y = tf32_rn(v.y - h.y) * lo_scale;
        l.z = tf32_rn(v.z - h.z) * lo_scale; l.w = tf32_rn(v.w - h.w) * lo_scale;
        X4[e] = h;
        L4[e] = l;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive_cta(&S.op_full[s]);
      return true;
    };
    auto make_q = [&](int i) -> bool {
      const int b = i & 1;
      if (!pipe_wait(S, &S.d1_full[b], static_cast<uint32_t>((i / 2) & 1), a.spin_limit, a.status)) return false;
      if (i >= 2 && !pipe_wait(S, &S.q_empty[b], static_cast<uint32_t>(((i / 2) - 1) & 1), a.spin_limit, a.status))
        return false;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int row = quarter * 32 + lane;  // TMEM lane = row of the tile
      float q[16];
      tmem_ld16(d1_addr(b) + (static_cast<uint32_t>(quarter * 32) << 16) + static_cast<uint32_t>(c0), q);
      const bool live = tile_row0(i) + row < rows;
#pragma unroll
      for (int c = 0; c < 16; ++c)
        if (!live || c0 + c >= a.kout) q[c] = 0.f;  // padding rows and columns of Q are zero
      unsigned char* qh = base + kOffQh + b * kPanelBytes;
      unsigned char* ql = base + kOffQl + b * kPanelBytes;
#pragma unroll
      for (int ch = 0; ch < 2; ++ch) {
        const int off = sw32b_chunk_offset(row, (c0 >> 3) + ch);
        const float* v = q + ch * 8;
        float4 h0 = make_float4(tf32_hi(v[0]), tf32_hi(v[1]), tf32_hi(v[2]), tf32_hi(v[3]));
        float4 h1 = make_float4(tf32_hi(v[4]), tf32_hi(v[5]), tf32_hi(v[6]), tf32_hi(v[7]));
        float4 l0 = make_float4(2.f * tf32_rn(v[0] - h0.x), 2.f * tf32_rn(v[1] - h0.y), 2.f * tf32_rn(v[2] - h0.z),
                                2.f * tf32_rn(v[3] - h0.w));
        float4 l1 = make_float4(2.f * tf32_rn(v[4] - h1.x), 2.f * tf32_rn(v[5] - h1.y), 2.f * tf32_rn(v[6] - h1.z),
                                2.f * tf32_rn(v[7] - h1.w));
        reinterpret_cast<float4*>(qh + off)[0] = h0;
        reinterpret_cast<float4*>(qh + off)[1] = h1;
        reinterpret_cast<float4*>(ql + off)[0] = l0;
        reinterpret_cast<float4*>(ql + off)[1] = l1;
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        mbar_arrive_cta(&S.d1_empty[b]);
        mbar_arrive_cta(&S.q_full[b]);
      }
      return true;
    };
    // Gram row of this thread's TMEM lane (M = 64: 16 rows per 32-lane quarter)
    const int grow = lane < 16 ? quarter * 16 + lane : -1;
    const bool has_cols = c0 < a.np;
    float grp[16], fh[16], fl[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      grp[j] = 0.f;
      fh[j] = 0.f;
      fl[j] = 0.f;
    }
    auto fold = [&]() {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        float s_, e_;
        two_sum(fh[j], grp[j], s_, e_);
        fh[j] = s_;
        fl[j] = __fadd_rn(fl[j], e_);
        grp[j] = 0.f;
      }
    };
    int grouped = 0;
    auto drain = [&](int i) -> bool {
      const int b = i & 1;
      if (!pipe_wait(S, &S.acc_full[b], static_cast<uint32_t>((i / 2) & 1), a.spin_limit, a.status)) return false;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (has_cols) {
        float sum[16], v[16];
        const uint32_t lanes = static_cast<uint32_t>(quarter * 32) << 16;
        tmem_ld16(acc_addr(b, 0) + lanes + static_cast<uint32_t>(c0), sum);
#pragma unroll 1
        for (int q = 1; q < kHiAcc; ++q) {
          tmem_ld16(acc_addr(b, q) + lanes + static_cast<uint32_t>(c0), v);
#pragma unroll
          for (int j = 0; j < 16; ++j) sum[j] = __fadd_rn(sum[j], v[j]);
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) grp[j] = __fadd_rn(grp[j], sum[j]);
        if (++grouped == kDrainGroup) {
          fold();
          grouped = 0;
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive_cta(&S.acc_empty[b]);
      return true;
    };
    bool ok = n == 0 || split(0);
    for (int i = 0; ok && i < n; ++i) {
      if (i + 1 < n && !split(i + 1)) break;
      if (pass2 && !make_q(i)) break;
      if (i >= 1 && !drain(i - 1)) break;
      if (i == n - 1) ok = drain(i);
    }
    fold();
    double* part = a.part + static_cast<int64_t>(blockIdx.x) * a.kout * a.kout;
    if (grow >= 0 && grow < a.kout && has_cols) {
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (c0 + j < a.kout) part[grow * a.kout + c0 + j] = static_cast<double>(fh[j]) + static_cast<double>(fl[j]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// ---------------------------------------------------------------------------
// Packed-operand engine: one M = 128 MMA per K step.
//
// A kind::tf32 MMA with M = 128 and K = 8 takes about 41, 49, 65 and 129
// tensor-pipe cycles at N = 32, 64, 128 and 256 (measured on this GPU), so
// the Gram is laid out to make each MMA as large as the tensor core allows.
// For a block of width kk in {4, 8, 16, 32}, R = 64 / kk consecutive rows are
// packed side by side into one 64-column "wide row", and the split parts
// form Z = [hi | lo] (128 columns, MN-major, 32-byte-atom 128-byte swizzle,
// four 32-column panels).
//
// Both passes accumulate D = Z^T H (N = 64: B is the hi half of Z), which
// holds, for each packed row position r, H_r^T H_r (hi lanes) and L_r^T H_r
// (lo lanes); the symmetrised sum H^T H + L^T H + H^T L takes the lo lanes
// twice, and L^T L is left out.  Pass 1 reads the packed rows straight from
// memory (the rows of a block are contiguous; hi = the raw value, which the
// tensor core truncates to TF32; |lo| < 2^-10 |v|), so its dropped term is at
// most 2^-20 of |v|^2 per product: the first factor only has to make Q well
// conditioned, and the second pass measures Q itself.
//
// Pass 2 forms Q = X W per tile of 128 rows in tensor memory with two MMAs
// per K step, X_hi [W_hi | W_lo] (N = 2 np) and X_lo W_hi (N = np), and Q is
// their sum X_hi W_hi + (X_hi W_lo + X_lo W_hi).  Q is split with hi = Q
// rounded to the nearest TF32 value and lo = Q - hi rounded to TF32, so the
// dropped L^T L term is below 2^-22 of |Q|^2 per product (2^-11 per lo
// part), under the FP32 rounding of the formation itself.
//
// Roles: a TMA producer warp, an MMA warp and three worker groups with loops
// of their own that meet only at mbarriers: split (the lo parts of each X
// tile; 2 warps in pass 2, 6 in pass 1), Q formation (pass 2: D1 from tensor
// memory into the packed operand; 4 warps, one per TMEM lane quarter) and
// drain (4 warps).  The MMA warp runs its loop warp-wide (warp votes keep the
// loop state and the descriptors uniform) and one elected lane issues the
// formations and Grams as their inputs become ready.  The producer prefetches
// the tile that will next reuse a stage into L2 when it loads the stage.
// Tensor memory: pass 1 two sets x two accumulators of 128 columns; pass 2
// two formation buffers of 2 np columns, two of np and two accumulators of
// 64.  Each drain thread adds its TMEM lane (one row of D) into float-float
// sums of the kk-wide row piece that belongs to its packed row position; the
// pieces are added in a fixed order at the end and each CTA's partial is
// written as float-float pairs.  Each pass is its own kernel (template P2),
// so that a kernel carries only the loops it runs.
constexpr int kPackStages = 3;  // pass-1 X stages (64 KB each)
constexpr int kP2Stages = 4;    // pass-2 X stages (32 KB each)
constexpr int kGroupWarps = 4;  // warps of the drain and Q-formation groups (one per TMEM lane quarter)
constexpr int kSplitWarps = 2;  // pass-2 split warps (pass 1 splits with these and the Q-formation group)
constexpr int kPackWarps = 2 + 2 * kGroupWarps + kSplitWarps;
constexpr int kPackThreads = 32 * kPackWarps;
constexpr int kP1Stage = 4 * kPanelBytes;         // pass 1: raw (2 panels) + lo (2 panels)
constexpr int kP2Stage = 2 * kPanelBytes;         // pass 2: raw (1 panel) + lo (1 panel)
constexpr int kP2Zq = kP2Stages * kP2Stage;       // 2 buffers x 4 panels x (64 rows x 128 B)
constexpr int kP2ZqBytes = 4 * 64 * 128;
constexpr int kP2Wh = kP2Zq + 2 * kP2ZqBytes;
constexpr int kP2Wl = kP2Wh + 32 * 128;
constexpr int kPackSmemBytes = (kPackStages * kP1Stage > kP2Wl + 32 * 128 ? kPackStages * kP1Stage : kP2Wl + 32 * 128) + 1024;

// N (4, 8, 16 or 32) consecutive TMEM columns of this thread's lane, no wait.
template <int N>
__device__ __forceinline__ void tmem_ld_nowait(uint32_t taddr, uint32_t (&r)[N]) {
  if constexpr (N == 4) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
  } else if constexpr (N == 8) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
  } else if constexpr (N == 16) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
  } else {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
        "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
  }
}

struct PackArgs {
  int k, kout, np, ksteps_f;
  int kk, rr;      // Gram width (k in pass 1, kout in pass 2) and rows per packed row (64 / kk)
  int64_t rows;
  const int64_t* rows_dev;
  const float* W;  // pass 2: W block base; nullptr for pass 1
  int wld;
  double* part;    // [grid][kout][kout]
  int32_t* status;
  int64_t spin_limit;
  int withhold;    // test-only: the producer never loads its first tile
  int64_t rows1;   // pass 2: rows of a second block (its own tensor map, the same W and Gram), 0: none
};

// Byte offset of column col (0..127) of packed row w in a Z panel set whose
// panels hold `wr` packed rows each (32-byte-atom 128-byte swizzle).
__device__ __forceinline__ int z_offset(int w, int col, int wr) {
  const int p = col >> 5, c = col & 31;
  return p * wr * 128 + w * 128 + ((((c >> 3) ^ (w & 3))) << 5) + ((c & 7) << 2);
}

// Pass-2 split of one landed X tile by the split warps (thread st: rows st,
// st + 32 kSplitWarps, ...): the CPR 16-byte chunks of each row that the
// formation reads (chunk c sits at c ^ (r mod 8) of the 128-byte swizzle;
// columns past k were zero-filled by the copy).  All loads are issued before
// any store; rows at or past `rows` are cleared in both parts.
template <int CPR>
__device__ __forceinline__ void split_rows_p2(float4* X4, float4* L4, int st, bool full, int64_t row0, int64_t rows) {
  constexpr int kRows = kTileRows / (32 * kSplitWarps);
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 v[kRows][CPR];
#pragma unroll
  for (int t = 0; t < kRows; ++t) {
    const int r = st + t * 32 * kSplitWarps;
#pragma unroll
    for (int c = 0; c < CPR; ++c) v[t][c] = X4[r * 8 + (c ^ (r & 7))];
  }
  if (full) {
#pragma unroll
    for (int t = 0; t < kRows; ++t) {
      const int r = st + t * 32 * kSplitWarps;
#pragma unroll
      for (int c = 0; c < CPR; ++c) {
        const float4 x = v[t][c];
        L4[r * 8 + (c ^ (r & 7))] = make_float4(tf32_rn(x.x - tf32_hi(x.x)), tf32_rn(x.y - tf32_hi(x.y)),
                                                tf32_rn(x.z - tf32_hi(x.z)), tf32_rn(x.w - tf32_hi(x.w)));
      }
    }
  } else {
#pragma unroll
    for (int t = 0; t < kRows; ++t) {
      const int r = st + t * 32 * kSplitWarps;
      const bool clear = row0 + r >= rows;
#pragma unroll
      for (int c = 0; c < CPR; ++c) {
        const int e = r * 8 + (c ^ (r & 7));
        const float4 x = v[t][c];
        if (clear) X4[e] = zero4;
        L4[e] = clear ? zero4
                      : make_float4(tf32_rn(x.x - tf32_hi(x.x)), tf32_rn(x.y - tf32_hi(x.y)),
                                    tf32_rn(x.z - tf32_hi(x.z)), tf32_rn(x.w - tf32_hi(x.w)));
      }
    }
  }
}

// P2 selects the pass at compile time (a.W != nullptr in pass 2), so that each
// kernel holds only its own pass's loops.
template <int KK, bool P2>
__device__ __forceinline__ void gram_pack_body(const CUtensorMap* tmx, const CUtensorMap* tmx1, const PackArgs& a,
                                               int cta, int G) {
  constexpr int RR = 64 / KK;  // rows per packed row
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ PipeSmem S;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr bool pass2 = P2;
  const int64_t rows = a.rows_dev ? *a.rows_dev : a.rows;
  // pass 1: tiles of 128 packed rows (128 R rows); pass 2: tiles of 128 rows,
  // those of the first block, then (rows1 > 0) those of the second from tmx1
  const int64_t tile_rows = pass2 ? kTileRows : static_cast<int64_t>(kTileRows) * a.rr;
  const int64_t nt0 = (rows + tile_rows - 1) / tile_rows;
  const int64_t ntiles_all = nt0 + (pass2 && a.rows1 > 0 ? (a.rows1 + tile_rows - 1) / tile_rows : 0);
  // tile t: its tensor map, first row within its block and the block's rows
  auto tile_src = [&](int64_t t, int64_t& r0, int64_t& lim) -> const CUtensorMap* {
    if (t < nt0) {
      r0 = t * tile_rows;
      lim = rows;
      return tmx;
    }
    r0 = (t - nt0) * tile_rows;
    lim = a.rows1;
    return tmx1;
  };
  const int n = ntiles_all > cta ? static_cast<int>((ntiles_all - 1 - cta) / G + 1) : 0;
  auto tile_index = [&](int i) -> int64_t { return static_cast<int64_t>(cta) + static_cast<int64_t>(i) * G; };
  const int nst = pass2 ? kP2Stages : kPackStages;  // X stages in flight
  const int stage_bytes = pass2 ? kP2Stage : kP1Stage;
  const int raw_bytes = stage_bytes / 2;  // the lo parts follow the raw (hi) parts of a stage
  const int wrq = kTileRows / a.rr;       // pass 2: packed rows of Q per tile
  // warps: 0 TMA, 1 MMA, 2-5 drain (D), 6-9 Q formation in pass 2 / split in pass 1, 10-11 split
  const int split_warp0 = pass2 ? 2 + 2 * kGroupWarps : 2 + kGroupWarps;
  const int split_warps = kPackWarps - split_warp0;

  if (tid == 0) {
    for (int q = 0; q < kPipeStages; ++q) {
      mbar_init(&S.tma_full[q], 1);
      mbar_init(&S.stage_empty[q], 1);
      mbar_init(&S.op_full[q], split_warps);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&S.d1_full[b], 1);
      mbar_init(&S.d1_empty[b], kGroupWarps);
      mbar_init(&S.q_full[b], kGroupWarps);
      mbar_init(&S.q_empty[b], 1);
      mbar_init(&S.acc_full[b], 1);
      mbar_init(&S.acc_empty[b], kGroupWarps);
    }
    mbar_init(&S.done, 1);
    S.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (pass2 && warp >= 2) {
    // [W_hi; W_lo]^T: 2 np rows x k, K-major 128-byte swizzle, zero padded;
    // the W_lo rows start at row np (a multiple of 16: whole 8-row atoms)
    constexpr int kStagers = kPackThreads - 64;
    const int wt = tid - 64;
    unsigned char* wb = base + kP2Wh;
    for (int e = wt; e < 2 * 32 * 32; e += kStagers) reinterpret_cast<float*>(wb)[e] = 0.f;
    asm volatile("bar.sync 1, %0;" ::"n"(kStagers) : "memory");
    for (int e = wt; e < a.kout * a.k; e += kStagers) {
      const int nn = e / a.k, kc = e - nn * a.k;
      const float v = (kc <= nn) ? a.W[static_cast<int64_t>(kc) * a.wld + nn] : 0.f;  // W upper triangular
      const float h = tf32_hi(v);
      *reinterpret_cast<float*>(wb + sw128_offset(nn, kc, 32 * 128)) = h;
      *reinterpret_cast<float*>(wb + sw128_offset(a.np + nn, kc, 32 * 128)) = tf32_rn(v - h);
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = S.tmem_base;
  // pass 2: D1[b] (2 np <= 64 columns: X_hi W_hi | X_hi W_lo), D1s[b] (np <= 32:
  // X_lo W_hi) and the Gram accumulators (64 columns each)
  auto d1_addr = [&](int b) { return tmem + static_cast<uint32_t>(b * 64); };
  auto d1s_addr = [&](int b) { return tmem + 128u + static_cast<uint32_t>(b * 32); };
  auto acc_addr = [&](int b, int q) {
    return pass2 ? tmem + 192u + static_cast<uint32_t>(b * 64) : tmem + static_cast<uint32_t>(b * 256 + q * 128);
  };
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  // The tensor core reads an FP32 operand as TF32 by ignoring its low 13
  // mantissa bits, so raw values serve as hi parts as they are; only the lo
  // parts (v - hi rounded to TF32) are written.
  auto lo_of = [](float4 v) {
    return make_float4(tf32_rn(v.x - tf32_hi(v.x)), tf32_rn(v.y - tf32_hi(v.y)), tf32_rn(v.z - tf32_hi(v.z)),
                       tf32_rn(v.w - tf32_hi(v.w)));
  };
  // Q = X W (TMEM lane qt = row of the tile) into the packed Gram operand: row
  // qt is packed row qt / R, position qt mod R (columns (qt mod R) KK + c).
  // A warp forms the rows of its lane quarter: the row of Q into registers,
  // X_hi W_hi + (X_hi W_lo + X_lo W_hi), D1 released as soon as it is read,
  // then the split parts into the Z buffer.
  auto q_form = [&](int i, int quarter) -> bool {
    constexpr int QH = KK;
    constexpr int cbase = 0;
    const int b = i & 1;
    const int qt = quarter * 32 + lane;
    const int w = qt / RR, c0 = (qt % RR) * KK + cbase;
    if (!warp_wait(S, &S.d1_full[b], static_cast<uint32_t>((i / 2) & 1), a.spin_limit, a.status)) return false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t lanes = (static_cast<uint32_t>(quarter * 32) << 16) + static_cast<uint32_t>(cbase);
    constexpr int QC = QH < 16 ? QH : 16;  // columns per TMEM read
    float v[QH];
#pragma unroll
    for (int cc = 0; cc < QH; cc += QC) {
      uint32_t qb[QC], qs[QC], qx[QC];
      tmem_ld_nowait<QC>(d1_addr(b) + lanes + static_cast<uint32_t>(cc), qb);
      tmem_ld_nowait<QC>(d1_addr(b) + lanes + static_cast<uint32_t>(a.np + cc), qs);
      tmem_ld_nowait<QC>(d1s_addr(b) + lanes + static_cast<uint32_t>(cc), qx);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int e = 0; e < QC; ++e)
        v[cc + e] = __fadd_rn(__uint_as_float(qb[e]), __fadd_rn(__uint_as_float(qs[e]), __uint_as_float(qx[e])));
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncwarp();
    if (lane == 0) mbar_arrive_cta(&S.d1_empty[b]);
    if (i >= 2 && !warp_wait(S, &S.q_empty[b], static_cast<uint32_t>(((i / 2) - 1) & 1), a.spin_limit, a.status))
      return false;
    int64_t qr0 = 0, qlim = 0;
    tile_src(tile_index(i), qr0, qlim);
    const bool live = qr0 + qt < qlim;
    unsigned char* zq = base + kP2Zq + b * kP2ZqBytes;
#pragma unroll
    for (int g = 0; g < QH / 4; ++g) {
      float4 h = zero4, l = zero4;
      if (live) {
        h = make_float4(tf32_rn(v[4 * g]), tf32_rn(v[4 * g + 1]), tf32_rn(v[4 * g + 2]), tf32_rn(v[4 * g + 3]));
        l = make_float4(tf32_rn(v[4 * g] - h.x), tf32_rn(v[4 * g + 1] - h.y), tf32_rn(v[4 * g + 2] - h.z),
                        tf32_rn(v[4 * g + 3] - h.w));
      }
      *reinterpret_cast<float4*>(zq + z_offset(w, c0 + 4 * g, wrq)) = h;
      *reinterpret_cast<float4*>(zq + z_offset(w, 64 + c0 + 4 * g, wrq)) = l;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    if (lane == 0) mbar_arrive_cta(&S.q_full[b]);
    return true;
  };

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int issued = 0;
      for (int i = 0; i < n; ++i) {
        const int s = i % nst;
        if (i >= nst && !pipe_wait(S, &S.stage_empty[s], static_cast<uint32_t>(((i / nst) - 1) & 1), a.spin_limit,
                                   a.status))
          break;
        if (a.withhold && i == 0) continue;  // the workers' bounded wait for this tile runs out
        unsigned char* dst = base + s * stage_bytes;
        const int y = static_cast<int>(tile_index(i) * kTileRows);
        if (pass2) {
          int64_t r0 = 0, lim = 0;
          const CUtensorMap* m = tile_src(tile_index(i), r0, lim);
          expect_tx(&S.tma_full[s], kPanelBytes);
          tma_load_2d(dst, m, 0, static_cast<int>(r0), &S.tma_full[s]);
        } else {  // 128 packed rows x 64 columns: two 32-column panels
          expect_tx(&S.tma_full[s], 2 * kPanelBytes);
          tma_load_2d(dst, tmx, 0, y, &S.tma_full[s]);
          tma_load_2d(dst + kPanelBytes, tmx, 32, y, &S.tma_full[s]);
        }
        // the tile that will next reuse this stage goes to L2 now, so that its
        // copy, issued when the stage frees, does not wait on HBM
        if (i + nst < n) {
          if (pass2) {
            int64_t r0 = 0, lim = 0;
            const CUtensorMap* m = tile_src(tile_index(i + nst), r0, lim);
            tma_prefetch_2d(m, 0, static_cast<int>(r0));
          } else {
            const int yp = static_cast<int>(tile_index(i + nst) * kTileRows);
            tma_prefetch_2d(tmx, 0, yp);
            tma_prefetch_2d(tmx, 32, yp);
          }
        }
        issued = i + 1;
      }
      for (int i = issued > nst ? issued - nst : 0; i < issued; ++i)
        if (!(a.withhold && i == 0))
          drain_wait(&S.tma_full[i % nst], static_cast<uint32_t>((i / nst) & 1), a.spin_limit, a.status);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issue
    const uint32_t idh = idesc_tf32(128, 64, 1);  // D = Z^T H: B is the first 64 columns of Z
    if (!pass2) {
      if (lane == 0) {
        for (int i = 0; i < n; ++i) {
          const int s = i % nst, b = i & 1;
          if (!pipe_wait(S, &S.op_full[s], static_cast<uint32_t>((i / nst) & 1), a.spin_limit, a.status)) break;
          if (i >= 2 && !pipe_wait(S, &S.acc_empty[b], static_cast<uint32_t>(((i / 2) - 1) & 1), a.spin_limit, a.status))
            break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          // Z = raw (hi) panels followed by the lo panels; K steps of 8 packed rows alternate accumulators
          const uint64_t dz = desc_mn_sw128_32b(smem_u32(base + s * stage_bytes), kPanelBytes);
#pragma unroll
          for (int ks = 0; ks < kTileRows / 8; ++ks)
            mma_tf32(acc_addr(b, ks & 1), dz + static_cast<uint64_t>(ks * 64), dz + static_cast<uint64_t>(ks * 64), idh,
                     ks >= 2 ? 1u : 0u);
          mma_commit(&S.stage_empty[s]);
          mma_commit(&S.acc_full[b]);
        }
        mma_commit(&S.done);
        drain_wait(&S.done, 0u, a.spin_limit, a.status);
      }
    } else {
      // Formations F(j) (D1[j & 1] = X_hi [W_hi | W_lo], D1s[j & 1] = X_lo W_hi)
      // and Grams G(i) are issued as their inputs become ready: F one or two
      // tiles ahead of G as the formation buffers allow.  Every barrier
      // tested here is at most one phase behind the phase tested (each test
      // follows the issue that consumed the previous phase), so the parity
      // tests are exact.  The loop gives up after spin_limit idle polls.
      // The shared-memory descriptors are computed once: their address
      // field holds bytes / 16, so the stages, the Z buffers and the K steps
      // (32 bytes of a K-major row, 1,024 bytes of 8 packed rows) are
      // constants added to a base descriptor, and the issue of a formation
      // or a Gram is a straight run of MMAs.  The whole warp runs the loop
      // and decides by warp votes, so the loop state and the descriptors
      // are warp-uniform; one elected lane issues every MMA and commit.
      const bool leader = elect_one();
      const uint32_t idf2 = idesc_tf32(128, 2 * a.np);  // X_hi [W_hi | W_lo]
      const uint32_t idf = idesc_tf32(128, a.np);       // X_lo W_hi
      const uint64_t dx0 = desc_kmajor_sw128(smem_u32(base));
      const uint64_t dwh = desc_kmajor_sw128(smem_u32(base + kP2Wh));
      const uint64_t dz0 = desc_mn_sw128_32b(smem_u32(base + kP2Zq), static_cast<uint32_t>(wrq * 128));
      const uint32_t idq = idesc_tf32(128, 64, 1);  // D = Z^T H: B is the first 64 columns of Z
      const int fsteps = a.ksteps_f, gsteps = wrq / 8;
      int nf = 0, ng = 0;
      int64_t idle = 0;
      while (ng < n) {
        bool progress = false;
        if (nf < n) {
          const int s = nf % nst, bd = nf & 1;
          const bool ready = mbar_test(&S.op_full[s], static_cast<uint32_t>((nf / nst) & 1)) &&
                             (nf < 2 || mbar_test(&S.d1_empty[bd], static_cast<uint32_t>(((nf / 2) - 1) & 1)));
          if (__all_sync(0xffffffffu, ready)) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t dah = dx0 + static_cast<uint64_t>((s * stage_bytes) >> 4);
            const uint64_t dal = dah + static_cast<uint64_t>(raw_bytes >> 4);
            const uint32_t d1 = d1_addr(bd), d1s = d1s_addr(bd);
            if (leader) {
#pragma unroll
              for (int ks = 0; ks < 4; ++ks)
                if (ks < fsteps) {
                  mma_tf32(d1, dah + 2u * ks, dwh + 2u * ks, idf2, ks > 0 ? 1u : 0u);
                  mma_tf32(d1s, dal + 2u * ks, dwh + 2u * ks, idf, ks > 0 ? 1u : 0u);
                }
              mma_commit(&S.stage_empty[s]);
              mma_commit(&S.d1_full[bd]);
            }
            __syncwarp();
            ++nf;
            progress = true;
          }
        }
        if (ng < nf) {
          const int b = ng & 1;
          const bool ready = mbar_test(&S.q_full[b], static_cast<uint32_t>((ng / 2) & 1)) &&
                             (ng < 2 || mbar_test(&S.acc_empty[b], static_cast<uint32_t>(((ng / 2) - 1) & 1)));
          if (__all_sync(0xffffffffu, ready)) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t dz = dz0 + static_cast<uint64_t>((b * kP2ZqBytes) >> 4);
            const uint32_t acc = acc_addr(b, 0);
            if (leader) {
              mma_tf32(acc, dz, dz, idq, 0u);
#pragma unroll
              for (int ks = 1; ks < 8; ++ks)
                if (ks < gsteps) mma_tf32(acc, dz + 64u * ks, dz + 64u * ks, idq, 1u);
              mma_commit(&S.q_empty[b]);
              mma_commit(&S.acc_full[b]);
            }
            __syncwarp();
            ++ng;
            progress = true;
          }
        }
        if (progress) {
          idle = 0;
        } else if (__any_sync(0xffffffffu, *reinterpret_cast<volatile int*>(&S.abort) != 0)) {
          break;
        } else if (++idle > a.spin_limit) {
          if (leader) set_status(a.status, kStatusTimeout);
          *reinterpret_cast<volatile int*>(&S.abort) = 1;
          break;
        } else if (idle > 8) {
          __nanosleep(32);  // leave the issue slots to the worker warps while nothing is ready
        }
      }
      if (leader) {  // the same lane that issued the MMAs: its commit tracks all of them
        mma_commit(&S.done);
        drain_wait(&S.done, 0u, a.spin_limit, a.status);
      }
    }
  } else if (warp >= split_warp0) {
    // ------------------------------------------------------------ split
    const int st = tid - 32 * split_warp0, nth = 32 * split_warps;
    for (int i = 0; i < n; ++i) {
      const int s = i % nst;
      if (!warp_wait(S, &S.tma_full[s], static_cast<uint32_t>((i / nst) & 1), a.spin_limit, a.status)) break;
      float4* X4 = reinterpret_cast<float4*>(base + s * stage_bytes);
      float4* L4 = reinterpret_cast<float4*>(base + s * stage_bytes + raw_bytes);
      const int64_t t0 = tile_index(i);
      int64_t r0 = 0, lim = 0;
      tile_src(t0, r0, lim);
      const bool full = r0 + tile_rows <= lim;  // no row of the tile lies past the end of its block
      if (!pass2) {
        // 2 panels of 128 packed rows (2,048 float4), loads before stores in batches of 4
        constexpr int kVec = kP1Stage / 2 / 16;
        for (int e0 = st; e0 < kVec; e0 += 4 * nth) {
          float4 v[4];
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            const int e = e0 + m * nth;
            v[m] = e < kVec ? X4[e] : zero4;
          }
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            const int e = e0 + m * nth;
            if (e < kVec) {
              bool clear = false;
              if (!full) {  // packed row w of panel p: the logical column gives the row inside the packed row
                const int p = e >> 10, w = (e & 1023) >> 3, slot = e & 7;
                const int col = p * 32 + (((slot >> 1) ^ (w & 3)) << 3) + ((slot & 1) << 2);
                clear = (t0 * kTileRows + w) * RR + col / KK >= rows;
              }
              if (clear) X4[e] = zero4;
              L4[e] = clear ? zero4 : lo_of(v[m]);
            }
          }
        }
      } else {
        // rows r = st, st + nth, ...: the 16-byte chunks c < 2 ceil(k / 8) the
        // formation reads (chunk c sits at c ^ (r mod 8) of the 128-byte
        // swizzle; columns past k are zero-filled by the copy)
        // (the chunk count is a compile-time constant of each case: straight-line code)
        switch (a.ksteps_f) {
          case 1: split_rows_p2<2>(X4, L4, st, full, r0, lim); break;
          case 2: split_rows_p2<4>(X4, L4, st, full, r0, lim); break;
          case 3: split_rows_p2<6>(X4, L4, st, full, r0, lim); break;
          default: split_rows_p2<8>(X4, L4, st, full, r0, lim); break;
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive_cta(&S.op_full[s]);
    }
  } else if (warp >= 2 + kGroupWarps) {
    // ------------------------------------------------------------ Q formation (pass 2)
    for (int i = 0; i < n; ++i)
      if (!q_form(i, warp & 3)) break;
  } else {
    // ------------------------------------------------------------ drain
    // This thread's TMEM lane is row i = 32 quarter + lane of D; within its
    // 64-row half it is position r * KK + a of a packed row.  Its piece of the
    // Gram row a sits in the 32-column chunk cb (hi columns) and 64 + cb (lo),
    // at columns (lane / KK) * KK ... + KK of the chunk: every KK-column group
    // of the chunk is loaded (warp-uniform addresses) and each lane keeps its
    // own.  Pass 1 has two accumulators (alternate K steps), added alike.
    const int quarter = warp & 3, gt = tid - 64;
    const int cb = (quarter & 1) * 32;
    const int mine = lane / KK;
    float grp[KK], fh[KK], fl[KK];
#pragma unroll
    for (int j = 0; j < KK; ++j) {
      grp[j] = 0.f;
      fh[j] = 0.f;
      fl[j] = 0.f;
    }
    int grouped = 0;
    auto fold = [&]() {
#pragma unroll
      for (int j = 0; j < KK; ++j) {
        float s_, e_;
        two_sum(fh[j], grp[j], s_, e_);
        fh[j] = s_;
        fl[j] = __fadd_rn(fl[j], e_);
        grp[j] = 0.f;
      }
    };
    for (int i = 0; i < n; ++i) {
      const int b = i & 1;
      if (!warp_wait(S, &S.acc_full[b], static_cast<uint32_t>((i / 2) & 1), a.spin_limit, a.status)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t lanes = static_cast<uint32_t>(quarter * 32) << 16;
      constexpr int C = 32 / KK;
      for (int q = 0; q < (pass2 ? 1 : 2); ++q) {
        const uint32_t acc = acc_addr(b, q) + lanes + static_cast<uint32_t>(cb);
        if constexpr (KK == 32) {  // the whole chunk is this lane's: two halves of 16 columns
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            uint32_t rh[16];
            tmem_ld_nowait<16>(acc + static_cast<uint32_t>(hh * 16), rh);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 16; ++j) grp[hh * 16 + j] = __fadd_rn(grp[hh * 16 + j], __uint_as_float(rh[j]));
          }
        } else {
          uint32_t rh[C][KK];
#pragma unroll
          for (int c = 0; c < C; ++c) tmem_ld_nowait<KK>(acc + static_cast<uint32_t>(c * KK), rh[c]);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int c = 0; c < C; ++c)
            if (c == mine) {
#pragma unroll
              for (int j = 0; j < KK; ++j) grp[j] = __fadd_rn(grp[j], __uint_as_float(rh[c][j]));
            }
        }
      }
      if (++grouped == kDrainGroup) {
        fold();
        grouped = 0;
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive_cta(&S.acc_empty[b]);
    }
    // pieces of each Gram row a: 2 halves x R positions, summed in a fixed order
    // in float-float (FP64 arithmetic is slow on this GPU: only the final entries are converted)
    asm volatile("bar.sync 2, %0;" ::"n"(32 * kGroupWarps) : "memory");
    float2* pieces = reinterpret_cast<float2*>(base);  // [128 lanes][32]; the stages are idle now
    fold();
    const int i128 = quarter * 32 + lane;
#pragma unroll
    for (int j = 0; j < KK; ++j) pieces[i128 * 32 + j] = make_float2(fh[j], fl[j]);
    asm volatile("bar.sync 2, %0;" ::"n"(32 * kGroupWarps) : "memory");
    double* part = a.part + static_cast<int64_t>(cta) * a.kout * a.kout;
    // pass 2 holds H^T H (hi lanes) and L^T H (lo lanes): the symmetrised sum
    // H^T H + L^T H + H^T L takes the lo lanes twice (exact scaling)
    const float lo_w = 2.f;
    auto gram_entry = [&](int ra, int cbb, float& h, float& l) {
      for (int half = 0; half < 2; ++half)
        for (int r = 0; r < RR; ++r) {
          float2 p = pieces[(half * 64 + r * KK + ra) * 32 + cbb];
          if (half == 1) p = make_float2(lo_w * p.x, lo_w * p.y);
          float s_, e_;
          two_sum(h, p.x, s_, e_);
          h = s_;
          l = __fadd_rn(l, __fadd_rn(e_, p.y));
        }
    };
    for (int e = gt; e < KK * KK; e += 32 * kGroupWarps) {  // upper triangle, symmetrised
      const int ra = e / KK, cbb = e - ra * KK;
      if (ra <= cbb) {
        float h = 0.f, l = 0.f;
        gram_entry(ra, cbb, h, l);
        gram_entry(cbb, ra, h, l);
        // the partial as a float-float pair (8 bytes, the slot of an FP64 value)
        reinterpret_cast<float2*>(part)[ra * a.kout + cbb] = make_float2(0.5f * h, 0.5f * l);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

template <int KK, bool P2>
__global__ void __launch_bounds__(kPackThreads, 1)
    gram_pack_kernel(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmx1, PackArgs a) {
  pdl_enter();
  gram_pack_body<KK, P2>(&tmx, &tmx1, a, blockIdx.x, gridDim.x);
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() { return tensor_map_encoder(); }

struct Geometry {
  TcArgs a;
  size_t smem;
};

__host__ __device__ inline int geo_take(int& off, int bytes) {
  const int o = off;
  off += (bytes + 1023) / 1024 * 1024;
  return o;
}

__host__ __device__ inline Geometry geometry(int k, int kout, bool pass2) {
  Geometry g{};
  TcArgs& a = g.a;
  a.k = k;
  a.kout = kout;
  a.kpanels = (k + 31) / 32;
  a.ksteps_f = (k + 7) / 8;
  a.np = (kout + 15) / 16 * 16;
  a.mg = kout <= 64 ? 64 : 128;
  a.qpanels = (kout + 31) / 32;
  a.wpanel_bytes = a.np * 128;
  int off = 0;
  const int xb = a.kpanels * kPanelBytes;
  a.off_x[0] = geo_take(off, xb);
  a.off_x[1] = geo_take(off, xb);
  a.off_xlo = geo_take(off, xb);
  a.off_wh = pass2 ? geo_take(off, a.kpanels * a.wpanel_bytes) : 0;
  a.off_wl = pass2 ? geo_take(off, a.kpanels * a.wpanel_bytes) : 0;
  a.off_qh = pass2 ? geo_take(off, a.qpanels * kPanelBytes) : 0;
  a.off_ql = pass2 ? geo_take(off, a.qpanels * kPanelBytes) : 0;
  a.alias = 0;
  if (pass2 && off + 1024 > 110 * 1024 && 2 * xb >= a.qpanels * kPanelBytes) {
    // too large for two CTAs per SM: X single-buffered (each tile loaded once
    // the previous tile's Gram is done) and Q's lo part over X and X's lo
    // part, which the formation has consumed by then
    off = 0;
    a.off_x[0] = geo_take(off, xb);
    a.off_xlo = geo_take(off, xb);  // (directly after X: one region of 2 xb bytes)
    a.off_x[1] = a.off_x[0];
    a.off_wh = geo_take(off, a.kpanels * a.wpanel_bytes);
    a.off_wl = geo_take(off, a.kpanels * a.wpanel_bytes);
    a.off_qh = geo_take(off, a.qpanels * kPanelBytes);
    a.off_ql = a.off_x[0];
    a.alias = 1;
  }
  g.smem = static_cast<size_t>(off) + 1024;  // + alignment of the dynamic base
  return g;
}

// ---- batched forms: one launch carries up to kTcJobs jobs (instance, Gram
// block) with their tensor maps as kernel arguments; job j owns CTAs
// [first[j], first[j+1]), and each CTA runs the engine's body over its
// job's tiles
constexpr int kTcJobs = 192;

struct TcBatch {
  CUtensorMap maps[kTcJobs];
  int32_t first[kTcJobs + 1];
  int32_t inst[kTcJobs];
  int8_t blk[kTcJobs];
  const Plan* plans;
  int njobs;
  int pass;
};

// Shape of Gram block b (0 head rows, 1 A tails, 2 B tails) in a pass.
struct BlockShape {
  const void* X;
  int k, kout;
  int64_t rows;
  const int64_t* rows_dev;
  const float* W;
};

__host__ __device__ inline BlockShape block_shape(const Plan& p, int pass, int b) {
  BlockShape sh{};
  if (b == 0) {
    sh.X = p.head;
    sh.k = p.n;
    sh.rows = p.t[0].m;
    sh.rows_dev = &p.hdr->num_runs[0];
  } else {
    sh.X = p.t[b - 1].tail;
    sh.k = p.t[b - 1].n;
    sh.rows = p.t[b - 1].m;
  }
  const int w0 = b == 2 ? p.n1 : 0;
  sh.kout = pass == 2 ? (b == 2 ? p.n2 : p.n) : sh.k;
  sh.W = pass == 2 ? p.Wf + static_cast<int64_t>(w0) * p.n + w0 : nullptr;
  return sh;
}

__device__ __forceinline__ PackArgs pack_args_of(const Plan& p, int pass, int b) {
  const BlockShape sh = block_shape(p, pass, b);
  PackArgs a{};
  const int kk = pass == 2 ? sh.kout : sh.k;
  a.k = sh.k;
  a.kout = sh.kout;
  a.np = (sh.kout + 15) / 16 * 16;
  a.ksteps_f = (sh.k + 7) / 8;
  a.kk = kk;
  a.rr = 64 / kk;
  a.rows = sh.rows;
  a.rows_dev = sh.rows_dev;
  a.W = sh.W;
  a.wld = p.n;
  a.part = p.gpart[b];
  a.status = &p.hdr->status;
  a.spin_limit = p.spin_limit;
  a.withhold = 0;
  return a;
}

__device__ __forceinline__ TcArgs tc_args_of(const Plan& p, int pass, int b) {
  const BlockShape sh = block_shape(p, pass, b);
  TcArgs a = geometry(sh.k, sh.kout, pass == 2).a;
  a.rows = sh.rows;
  a.rows_dev = sh.rows_dev;
  a.W = sh.W;
  a.wld = p.n;
  a.part = p.gpart[b];
  a.status = &p.hdr->status;
  a.spin_limit = p.spin_limit;
  return a;
}

__device__ __forceinline__ int tc_batch_job(const TcBatch& B, int cta) {
  int lo = 0, hi = B.njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (B.first[mid] <= cta)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

template <int KK, bool P2>
__global__ void __launch_bounds__(kPackThreads, 1) gram_pack_batched(const __grid_constant__ TcBatch B) {
  pdl_enter();
  const int j = tc_batch_job(B, blockIdx.x);
  const PackArgs a = pack_args_of(B.plans[B.inst[j]], B.pass, B.blk[j]);
  gram_pack_body<KK, P2>(&B.maps[j], &B.maps[j], a, blockIdx.x - B.first[j], B.first[j + 1] - B.first[j]);
}

template <int NP>
__global__ void __launch_bounds__(kTcThreads) gram_tc_batched(const __grid_constant__ TcBatch B) {
  pdl_enter();
  const int j = tc_batch_job(B, blockIdx.x);
  const TcArgs a = tc_args_of(B.plans[B.inst[j]], B.pass, B.blk[j]);
  gram_tc_body<NP>(&B.maps[j], a, blockIdx.x - B.first[j], B.first[j + 1] - B.first[j]);
}


// ---------------------------------------------------------------------------
// Tiled Gram of wide blocks: one CTA per (block, 128 x 128 upper tile pair
// (ti, tj), row split) accumulates C = X_i^T X_j over its rows in 3 x TF32,
// C = H_i^T H_j + (H_i^T L_j + L_i^T H_j): the large products and the two
// correction products go to separate tensor-memory accumulators (a truncated
// FP32 accumulator then loses bits only relative to what it holds), both
// double-buffered (4 x 128 of the 512 columns).  Per stage of 32 rows the
// producer copies the tiles' 32-column panels (32-byte-atom 128-byte swizzle:
// the MN-major operand layout), the split warps write the lo parts beside
// them, and the MMA warp issues 4 K steps x 3 MMAs (M = N = 128, K = 8).
// Every two stages (64 rows) the drain warps add both accumulators into FP32
// registers; every 8 drains (512 rows) and at the end each drain thread adds
// its 64 entries of the tile into the job's FP64 partial (its own row, so no
// two threads touch one entry).
constexpr int kWtRows = 32;                        // rows per stage
constexpr int kWtStages = 3;
constexpr int kWtPanel = kWtRows * 128;            // 32 rows x 32 columns (4 KB)
constexpr int kWtTileBytes = 4 * kWtPanel;         // one 128-column tile of a stage
constexpr int kWtStage = 4 * kWtTileBytes;         // hi of tiles i, j; lo of tiles i, j
constexpr int kWtSmem = kWtStages * kWtStage + 1024;
constexpr int kWtDrainWarps = 8;                   // two per TMEM lane quarter, 64 columns each
constexpr int kWtSplitWarps = 4;
constexpr int kWtWarps = 2 + kWtDrainWarps + kWtSplitWarps;
constexpr int kWtThreads = 32 * kWtWarps;
constexpr int kWtFold = 8;                         // drains per FP64 fold

struct WideTcArgs {
  CUtensorMap map[3];
  WideTcBlock b[3];
  int job0[3];
  double* part;
  int32_t* status;
  int64_t spin_limit;
};

// One job of the tile Gram: block B (its rows in tensor map `map`), partials
// of all its jobs from part_all.
__device__ __forceinline__ void wide_gram_tc_body(const WideTcBlock& B, const CUtensorMap* map, int job,
                                                  double* part_all, int32_t* status, int64_t spin_limit) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ PipeSmem S;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tile = job / B.splits, split = job - tile * B.splits;
  int ti = 0, len = B.tiles, t = tile;  // upper tile pair (ti <= tj), row-major over the upper triangle
  while (t >= len) {
    t -= len;
    ++ti;
    --len;
  }
  const int tj = ti + t;
  const bool two = ti != tj;
  const int64_t rows_all = B.rows_dev ? (*B.rows_dev < B.rows ? *B.rows_dev : B.rows) : B.rows;
  const int64_t r0 = static_cast<int64_t>(split) * B.split_rows;
  int64_t r1 = r0 + B.split_rows;
  if (r1 > rows_all) r1 = rows_all;
  const int nst = r1 > r0 ? static_cast<int>((r1 - r0 + kWtRows - 1) / kWtRows) : 0;
  const int ngroups = (nst + 1) / 2;
  double* part = part_all + static_cast<int64_t>(job) * kWideTcTile * kWideTcTile;

  if (tid == 0) {
    for (int q = 0; q < kWtStages; ++q) {
      mbar_init(&S.tma_full[q], 1);
      mbar_init(&S.stage_empty[q], 1);
      mbar_init(&S.op_full[q], kWtSplitWarps);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&S.acc_full[b], 1);
      mbar_init(&S.acc_empty[b], kWtDrainWarps);
    }
    mbar_init(&S.done, 1);
    S.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = S.tmem_base;
  const int tile_bytes = (two ? 2 : 1) * kWtTileBytes;  // hi bytes copied per stage

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int issued = 0;
      for (int s = 0; s < nst; ++s) {
        const int q = s % kWtStages;
        if (s >= kWtStages && !pipe_wait(S, &S.stage_empty[q], static_cast<uint32_t>(((s / kWtStages) - 1) & 1),
                                         spin_limit, status))
          break;
        unsigned char* dst = base + q * kWtStage;
        const int y = static_cast<int>(r0 + static_cast<int64_t>(s) * kWtRows);
        expect_tx(&S.tma_full[q], static_cast<uint32_t>(tile_bytes));
        for (int p = 0; p < 4; ++p) tma_load_2d(dst + p * kWtPanel, map, ti * kWideTcTile + 32 * p, y, &S.tma_full[q]);
        if (two)
          for (int p = 0; p < 4; ++p)
            tma_load_2d(dst + kWtTileBytes + p * kWtPanel, map, tj * kWideTcTile + 32 * p, y, &S.tma_full[q]);
        issued = s + 1;
      }
      for (int s = issued > kWtStages ? issued - kWtStages : 0; s < issued; ++s)
        drain_wait(&S.tma_full[s % kWtStages], static_cast<uint32_t>((s / kWtStages) & 1), spin_limit, status);
    }
  } else if (warp >= 2 + kWtDrainWarps) {
    // ------------------------------------------------------------ split
    // lo = TF32(x - hi) beside each copied panel; rows at or past the job's
    // end (the block's last rows, or rows past the device row count) are
    // cleared in both parts
    const int st = tid - 32 * (2 + kWtDrainWarps);
    const int nf4 = tile_bytes / 16;
    for (int s = 0; s < nst; ++s) {
      const int q = s % kWtStages;
      if (!warp_wait(S, &S.tma_full[q], static_cast<uint32_t>((s / kWtStages) & 1), spin_limit, status)) break;
      float4* X4 = reinterpret_cast<float4*>(base + q * kWtStage);
      float4* L4 = reinterpret_cast<float4*>(base + q * kWtStage + 2 * kWtTileBytes);
      const int64_t valid = r1 - (r0 + static_cast<int64_t>(s) * kWtRows);  // rows of this stage in the job
      for (int e0 = st; e0 < nf4; e0 += 4 * 32 * kWtSplitWarps) {
        float4 v[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const int e = e0 + m * 32 * kWtSplitWarps;
          v[m] = e < nf4 ? X4[e] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const int e = e0 + m * 32 * kWtSplitWarps;
          if (e < nf4) {
            const int row = (e & (kWtPanel / 16 - 1)) >> 3;  // 8 float4 per 128-byte row of a panel
            if (row >= valid) {
              X4[e] = make_float4(0.f, 0.f, 0.f, 0.f);
              L4[e] = make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
              const float4 x = v[m];
              L4[e] = make_float4(tf32_rn(x.x - tf32_hi(x.x)), tf32_rn(x.y - tf32_hi(x.y)), tf32_rn(x.z - tf32_hi(x.z)),
                                  tf32_rn(x.w - tf32_hi(x.w)));
            }
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive_cta(&S.op_full[q]);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issue
    // warp-wide loop (every wait answers all lanes alike), one elected issuer
    const bool leader = elect_one();
    const uint32_t idg = idesc_tf32(128, 128, 1);
    const uint64_t d0 = desc_mn_sw128_32b(smem_u32(base), kWtPanel);
    for (int s = 0; s < nst; ++s) {
      const int q = s % kWtStages, g = s / 2, b = g & 1;
      if (!warp_wait(S, &S.op_full[q], static_cast<uint32_t>((s / kWtStages) & 1), spin_limit, status)) break;
      if ((s & 1) == 0 && g >= 2 &&
          !warp_wait(S, &S.acc_empty[b], static_cast<uint32_t>(((g / 2) - 1) & 1), spin_limit, status))
        break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t dhi = d0 + static_cast<uint64_t>((q * kWtStage) >> 4);
      const uint64_t dhj = two ? dhi + static_cast<uint64_t>(kWtTileBytes >> 4) : dhi;
      const uint64_t dli = dhi + static_cast<uint64_t>((2 * kWtTileBytes) >> 4);
      const uint64_t dlj = dhj + static_cast<uint64_t>((2 * kWtTileBytes) >> 4);
      const uint32_t big = tmem + static_cast<uint32_t>(b * 256), small = big + 128u;
      if (leader) {
#pragma unroll
        for (int k = 0; k < kWtRows / 8; ++k) {  // K steps of 8 rows (1 KB of each panel)
          const uint32_t acc = ((s & 1) == 0 && k == 0) ? 0u : 1u;
          const uint64_t o = static_cast<uint64_t>(64 * k);
          mma_tf32(big, dhi + o, dhj + o, idg, acc);
          mma_tf32(small, dhi + o, dlj + o, idg, acc);
          mma_tf32(small, dli + o, dhj + o, idg, 1u);
        }
        mma_commit(&S.stage_empty[q]);
        if ((s & 1) == 1 || s == nst - 1) mma_commit(&S.acc_full[b]);
      }
      __syncwarp();
    }
    if (leader) {  // the lane that issued the MMAs: its commit tracks all of them
      mma_commit(&S.done);
      drain_wait(&S.done, 0u, spin_limit, status);
    }
  } else {
    // ------------------------------------------------------------ drain
    // thread: row 32 quarter + lane of the tile, columns [64 half, 64 half + 64)
    const int dw = warp - 2, quarter = warp & 3, half = dw >> 2;
    const int row = quarter * 32 + lane;
    const uint32_t lanes = (static_cast<uint32_t>(quarter * 32) << 16) + static_cast<uint32_t>(64 * half);
    double* prow = part + static_cast<int64_t>(row) * kWideTcTile + 64 * half;
    float acc[64];
#pragma unroll
    for (int e = 0; e < 64; ++e) acc[e] = 0.f;
    bool first = true;
    // the first fold stores, later ones add without reading back (each entry
    // belongs to this thread alone, so its additions keep program order)
    auto fold = [&]() {
      // (each conversion sits with its store, so that one FP64 value is live at a time)
      if (first) {
#pragma unroll
        for (int e = 0; e < 32; ++e)
          asm volatile("{ .reg .f64 a, b; cvt.f64.f32 a, %1; cvt.f64.f32 b, %2; st.global.v2.f64 [%0], {a, b}; }" ::"l"(
                           prow + 2 * e),
                       "f"(acc[2 * e]), "f"(acc[2 * e + 1])
                       : "memory");
      } else {
#pragma unroll
        for (int e = 0; e < 64; ++e)
          asm volatile("{ .reg .f64 a; cvt.f64.f32 a, %1; red.global.add.f64 [%0], a; }" ::"l"(prow + e), "f"(acc[e])
                       : "memory");
      }
#pragma unroll
      for (int e = 0; e < 64; ++e) acc[e] = 0.f;
      first = false;
    };
    int since = 0;
    for (int g = 0; g < ngroups; ++g) {
      const int b = g & 1;
      if (!warp_wait(S, &S.acc_full[b], static_cast<uint32_t>((g / 2) & 1), spin_limit, status)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t big = tmem + static_cast<uint32_t>(b * 256) + lanes, small = big + 128u;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        uint32_t hb[16], hs[16];
        tmem_ld_nowait<16>(big + static_cast<uint32_t>(16 * c), hb);
        tmem_ld_nowait<16>(small + static_cast<uint32_t>(16 * c), hs);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int e = 0; e < 16; ++e)
          acc[16 * c + e] = __fadd_rn(acc[16 * c + e], __fadd_rn(__uint_as_float(hb[e]), __uint_as_float(hs[e])));
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive_cta(&S.acc_empty[b]);
      if (++since == kWtFold) {
        fold();
        since = 0;
      }
    }
    if (first || since > 0) fold();  // (a job without rows writes zeros)
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// Entry of a table launch: the highest i with job0[i] <= x (entries own
// [job0[i], job0[i + 1]) CTAs).
__device__ __forceinline__ int table_entry(const int32_t* __restrict__ job0, int nb, int x) {
  int lo = 0, hi = nb - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (job0[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Tensor maps that reach a launch through device memory (written there by an
// earlier kernel): order those generic-proxy writes before this thread's
// tensor copies.
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap* m) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(m) : "memory");
}

__global__ void __launch_bounds__(kWtThreads, 1) wide_gram_tc_kernel(const __grid_constant__ WideTcArgs A) {
  pdl_enter();
  int bi = 0;
  while (bi < 2 && static_cast<int>(blockIdx.x) >= A.job0[bi] + A.b[bi].njobs) ++bi;
  const WideTcBlock& B = A.b[bi];
  wide_gram_tc_body(B, &A.map[bi], static_cast<int>(blockIdx.x) - A.job0[bi], A.part + B.pbase, A.status,
                    A.spin_limit);
}

__global__ void __launch_bounds__(kWtThreads, 1)
    wide_gram_tc_table_kernel(const WideTcEntry* __restrict__ E, const int32_t* __restrict__ job0, int nb,
                              int64_t spin_limit) {
  pdl_enter();
  const int bi = table_entry(job0, nb, static_cast<int>(blockIdx.x));
  const WideTcEntry& e = E[bi];
  tensormap_acquire(&e.map);
  wide_gram_tc_body(e.b, &e.map, static_cast<int>(blockIdx.x) - job0[bi], e.b.part, e.b.status, spin_limit);
}

// ---------------------------------------------------------------------------
// Tensor-core formation of wide blocks: Q = X W[w0:w0+k, w0:w0+kout] in
// 3 x TF32, Q = X_hi W_hi + (X_hi W_lo + X_lo W_hi).  One CTA per (block,
// 128-column tile ct of Q, range of 128-row tiles).  A stage is one 32-column
// K panel: the X panel (128 rows, K-major 128-byte swizzle) and its lo part,
// and the panel of W^T (128 output columns) with its lo part, prepared once
// per pass.  K panels that meet only zeros of the upper-triangular W
// (features past the tile's last column) are skipped.  Every two panels the
// drain warps add the two accumulators (large products, corrections) into
// FP32 registers; at the end of a row tile they store its rows of Q.
constexpr int kWfPanel = 128 * 128;   // 128 rows x 32 columns (16 KB)
constexpr int kWfStage = 4 * kWfPanel;  // X, X lo, W^T, W^T lo
constexpr int kWfSmem = kWtStages * kWfStage + 1024;

struct WideFormArgs {
  CUtensorMap xmap[3];
  CUtensorMap wmap, wlmap;
  WideFormBlock b[3];
  int job0[3];
  int32_t* status;
  int64_t spin_limit;
};

// W^T and its TF32 lo parts (W upper triangular: W^T[c][f] = W[f][c] for f <= c).
__device__ __forceinline__ void wide_form_prep_at(const float* W, int n, float* WT, float* WTlo, int64_t e) {
  if (e >= static_cast<int64_t>(n) * n) return;
  const int c = static_cast<int>(e / n), f = static_cast<int>(e - static_cast<int64_t>(c) * n);
  const float v = f <= c ? W[static_cast<int64_t>(f) * n + c] : 0.f;
  WT[e] = v;
  WTlo[e] = tf32_rn(v - tf32_hi(v));
}

__global__ void wide_form_prep_kernel(const float* W, int n, float* WT, float* WTlo) {
  pdl_enter();
  wide_form_prep_at(W, n, WT, WTlo, static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x);
}

// One job of the formation: block B, its X rows in xmap, W^T and its lo parts
// in wmap and wlmap.
__device__ __forceinline__ void wide_form_tc_body(const WideFormBlock& B, const CUtensorMap* xmap,
                                                  const CUtensorMap* wmap, const CUtensorMap* wlmap, int job,
                                                  int32_t* status, int64_t spin_limit) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ PipeSmem S;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ct = job / B.splits, split = job - ct * B.splits;
  const int64_t rows_all = B.rows_dev ? (*B.rows_dev < B.rows ? *B.rows_dev : B.rows) : B.rows;
  const int nrt_all = static_cast<int>((rows_all + 127) / 128);
  const int rt0 = split * B.rt_per_split;
  int nrt = nrt_all - rt0;
  if (nrt > B.rt_per_split) nrt = B.rt_per_split;
  if (nrt < 0) nrt = 0;
  int nkp = (B.k + 31) / 32;
  if (nkp > 4 * ct + 4) nkp = 4 * ct + 4;  // W^T rows of the tile end at column 128 ct + 127
  const int nst = nrt * nkp;
  const int gpr = (nkp + 1) / 2;  // drain groups per row tile
  const int ngroups = nrt * gpr;

  if (tid == 0) {
    for (int q = 0; q < kWtStages; ++q) {
      mbar_init(&S.tma_full[q], 1);
      mbar_init(&S.stage_empty[q], 1);
      mbar_init(&S.op_full[q], kWtSplitWarps);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&S.acc_full[b], 1);
      mbar_init(&S.acc_empty[b], kWtDrainWarps);
    }
    mbar_init(&S.done, 1);
    S.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = S.tmem_base;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int issued = 0;
      for (int s = 0; s < nst; ++s) {
        const int q = s % kWtStages, rt = rt0 + s / nkp, kp = s % nkp;
        if (s >= kWtStages && !pipe_wait(S, &S.stage_empty[q], static_cast<uint32_t>(((s / kWtStages) - 1) & 1),
                                         spin_limit, status))
          break;
        unsigned char* dst = base + q * kWfStage;
        expect_tx(&S.tma_full[q], static_cast<uint32_t>(3 * kWfPanel));
        tma_load_2d(dst, xmap, 32 * kp, 128 * rt, &S.tma_full[q]);
        tma_load_2d(dst + 2 * kWfPanel, wmap, B.w0 + 32 * kp, B.w0 + 128 * ct, &S.tma_full[q]);
        tma_load_2d(dst + 3 * kWfPanel, wlmap, B.w0 + 32 * kp, B.w0 + 128 * ct, &S.tma_full[q]);
        issued = s + 1;
      }
      for (int s = issued > kWtStages ? issued - kWtStages : 0; s < issued; ++s)
        drain_wait(&S.tma_full[s % kWtStages], static_cast<uint32_t>((s / kWtStages) & 1), spin_limit, status);
    }
  } else if (warp >= 2 + kWtDrainWarps) {
    // ------------------------------------------------------------ split (X lo; rows past the block's end cleared)
    const int st = tid - 32 * (2 + kWtDrainWarps);
    constexpr int NT = 32 * kWtSplitWarps;
    for (int s = 0; s < nst; ++s) {
      const int q = s % kWtStages, rt = rt0 + s / nkp;
      if (!warp_wait(S, &S.tma_full[q], static_cast<uint32_t>((s / kWtStages) & 1), spin_limit, status)) break;
      float4* X4 = reinterpret_cast<float4*>(base + q * kWfStage);
      float4* L4 = reinterpret_cast<float4*>(base + q * kWfStage + kWfPanel);
      const int64_t valid = rows_all - static_cast<int64_t>(rt) * 128;
      for (int e0 = st; e0 < kWfPanel / 16; e0 += 4 * NT) {
        float4 v[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) v[m] = X4[e0 + m * NT];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const int e = e0 + m * NT;
          if ((e >> 3) >= valid) {  // row e / 8 of the panel (128-byte rows)
            X4[e] = make_float4(0.f, 0.f, 0.f, 0.f);
            L4[e] = make_float4(0.f, 0.f, 0.f, 0.f);
          } else {
            const float4 x = v[m];
            L4[e] = make_float4(tf32_rn(x.x - tf32_hi(x.x)), tf32_rn(x.y - tf32_hi(x.y)), tf32_rn(x.z - tf32_hi(x.z)),
                                tf32_rn(x.w - tf32_hi(x.w)));
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive_cta(&S.op_full[q]);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issue (warp-wide loop, one elected issuer)
    const bool leader = elect_one();
    const uint32_t idf = idesc_tf32(128, 128);  // both operands K-major
    const uint64_t d0 = desc_kmajor_sw128(smem_u32(base));
    for (int s = 0; s < nst; ++s) {
      const int q = s % kWtStages, kp = s % nkp;
      const int g = (s / nkp) * gpr + kp / 2, b = g & 1;
      const bool first_of_group = (kp & 1) == 0;
      const bool last_of_group = (kp & 1) == 1 || kp == nkp - 1;
      if (!warp_wait(S, &S.op_full[q], static_cast<uint32_t>((s / kWtStages) & 1), spin_limit, status)) break;
      if (first_of_group && g >= 2 &&
          !warp_wait(S, &S.acc_empty[b], static_cast<uint32_t>(((g / 2) - 1) & 1), spin_limit, status))
        break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t dx = d0 + static_cast<uint64_t>((q * kWfStage) >> 4);
      const uint64_t dxl = dx + static_cast<uint64_t>(kWfPanel >> 4);
      const uint64_t dw = dx + static_cast<uint64_t>((2 * kWfPanel) >> 4);
      const uint64_t dwl = dx + static_cast<uint64_t>((3 * kWfPanel) >> 4);
      const uint32_t big = tmem + static_cast<uint32_t>(b * 256), small = big + 128u;
      if (leader) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {  // K steps of 8 columns (32 bytes of each 128-byte row)
          const uint32_t acc = (first_of_group && k == 0) ? 0u : 1u;
          const uint64_t o = static_cast<uint64_t>(2 * k);
          mma_tf32(big, dx + o, dw + o, idf, acc);
          mma_tf32(small, dx + o, dwl + o, idf, acc);
          mma_tf32(small, dxl + o, dw + o, idf, 1u);
        }
        mma_commit(&S.stage_empty[q]);
        if (last_of_group) mma_commit(&S.acc_full[b]);
      }
      __syncwarp();
    }
    if (leader) {
      mma_commit(&S.done);
      drain_wait(&S.done, 0u, spin_limit, status);
    }
  } else {
    // ------------------------------------------------------------ drain and store
    // thread: row 32 quarter + lane of the row tile, columns [64 half, 64 half + 64) of the column tile
    const int dw = warp - 2, quarter = warp & 3, half = dw >> 2;
    const int row = quarter * 32 + lane;
    const uint32_t lanes = (static_cast<uint32_t>(quarter * 32) << 16) + static_cast<uint32_t>(64 * half);
    const int c0 = ct * 128 + 64 * half;
    float acc[64];
#pragma unroll
    for (int e = 0; e < 64; ++e) acc[e] = 0.f;
    for (int g = 0; g < ngroups; ++g) {
      const int b = g & 1;
      if (!warp_wait(S, &S.acc_full[b], static_cast<uint32_t>((g / 2) & 1), spin_limit, status)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t big = tmem + static_cast<uint32_t>(b * 256) + lanes, small = big + 128u;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        uint32_t hb[16], hs[16];
        tmem_ld_nowait<16>(big + static_cast<uint32_t>(16 * c), hb);
        tmem_ld_nowait<16>(small + static_cast<uint32_t>(16 * c), hs);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int e = 0; e < 16; ++e)
          acc[16 * c + e] = __fadd_rn(acc[16 * c + e], __fadd_rn(__uint_as_float(hb[e]), __uint_as_float(hs[e])));
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive_cta(&S.acc_empty[b]);
      if ((g % gpr) == gpr - 1) {  // the row tile is complete: its row of Q, then a fresh sum
        const int64_t r = static_cast<int64_t>(rt0 + g / gpr) * 128 + row;
        if (r < rows_all) {
          float* qrow = B.Q + r * B.kout;
#pragma unroll
          for (int e = 0; e < 64; e += 4)
            if (c0 + e < B.kout)
              *reinterpret_cast<float4*>(qrow + c0 + e) = make_float4(acc[e], acc[e + 1], acc[e + 2], acc[e + 3]);
        }
#pragma unroll
        for (int e = 0; e < 64; ++e) acc[e] = 0.f;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

__global__ void __launch_bounds__(kWtThreads, 1) wide_form_tc_kernel(const __grid_constant__ WideFormArgs A) {
  pdl_enter();
  int bi = 0;
  while (bi < 2 && static_cast<int>(blockIdx.x) >= A.job0[bi] + A.b[bi].njobs) ++bi;
  wide_form_tc_body(A.b[bi], &A.xmap[bi], &A.wmap, &A.wlmap, static_cast<int>(blockIdx.x) - A.job0[bi], A.status,
                    A.spin_limit);
}

__global__ void __launch_bounds__(kWtThreads, 1)
    wide_form_tc_table_kernel(const WideFormEntry* __restrict__ E, const int32_t* __restrict__ job0, int nb,
                              int64_t spin_limit) {
  pdl_enter();
  const int bi = table_entry(job0, nb, static_cast<int>(blockIdx.x));
  const WideFormEntry& e = E[bi];
  tensormap_acquire(&e.xmap);
  tensormap_acquire(&e.wmap);
  tensormap_acquire(&e.wlmap);
  wide_form_tc_body(e.b, &e.xmap, &e.wmap, &e.wlmap, static_cast<int>(blockIdx.x) - job0[bi], e.b.status,
                    spin_limit);
}

__global__ void wide_prep_table_kernel(const WidePrepEntry* __restrict__ E, const int32_t* __restrict__ cta0,
                                       int nb) {
  pdl_enter();
  const int bi = table_entry(cta0, nb, static_cast<int>(blockIdx.x));
  const WidePrepEntry& e = E[bi];
  wide_form_prep_at(e.W, e.n, e.WT, e.WTlo,
                    static_cast<int64_t>(static_cast<int>(blockIdx.x) - cta0[bi]) * blockDim.x + threadIdx.x);
}

}  // namespace

// The packed engine writes symmetrised upper-triangle partials; the others
// write P with G = (P + P^T) / 2.
bool gram_tc_packs(int k, int kout, bool pass2) {
  const int kk = pass2 ? kout : k;
  return (kk == 4 || kk == 8 || kk == 16 || kk == 32) && k <= 32;
}

// The tensor-core engine handles a Gram block when TMA can address X
// (k a multiple of 4) and the block fits the 64-column tile.
bool wide_tc_eligible(const float* X, int64_t ld, int kout) {
  return X != nullptr && kout >= 1 && ld >= kout && ld % 4 == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0 &&
         encoder() != nullptr;
}

namespace {

// The rows of a tile-Gram block: 32-column by kWtRows-row boxes (32-byte
// atoms of the 128-byte swizzle, the MN-major operand layout).
bool encode_wt_map(CUtensorMap* m, const WideTcBlock& b) {
  if (!wide_tc_eligible(b.X, b.ld, b.kout)) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(b.kout), static_cast<cuuint64_t>(b.rows > 0 ? b.rows : 1)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(b.ld) * 4};
  cuuint32_t box[2] = {32, static_cast<cuuint32_t>(kWtRows)};
  cuuint32_t es[2] = {1, 1};
  return encoder()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(b.X), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B_ATOM_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Operands of the formation: 32-column by 128-row boxes, K-major 128-byte swizzle.
bool encode_wf_map(CUtensorMap* m, const float* p, int64_t inner, int64_t outer, int64_t ld) {
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(inner), static_cast<cuuint64_t>(outer > 0 ? outer : 1)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * 4};
  cuuint32_t box[2] = {32, 128};
  cuuint32_t es[2] = {1, 1};
  return encoder()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(p), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool form_block_ok(const WideFormBlock& b) {
  return wide_tc_eligible(b.X, b.ldx, b.k) && b.kout % 4 == 0 && (reinterpret_cast<uintptr_t>(b.Q) & 15) == 0;
}

bool form_w_ok(const float* WT, const float* WTlo, int n) {
  return n % 4 == 0 && wide_tc_eligible(WT, n, n) && wide_tc_eligible(WTlo, n, n);
}

// Dynamic shared memory above 48 KB, granted once per device and kernel.
template <typename K>
cudaError_t grant_smem(K kern, int bytes, int* granted) {
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev >= 0 && dev < 64 && granted[dev]) return cudaSuccess;
  err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (err == cudaSuccess && dev >= 0 && dev < 64) granted[dev] = 1;
  return err;
}

}  // namespace

cudaError_t launch_wide_gram_tc(const WideTcBlock b[3], double* part, int32_t* status, int64_t spin_limit,
                                cudaStream_t s) {
  WideTcArgs a;
  std::memset(&a, 0, sizeof(a));
  int jobs = 0;
  for (int i = 0; i < 3; ++i) {
    a.b[i] = b[i];
    a.job0[i] = jobs;
    jobs += b[i].njobs;
    if (b[i].njobs == 0) continue;
    if (!encode_wt_map(&a.map[i], b[i])) return cudaErrorInvalidValue;
  }
  if (jobs == 0) return cudaSuccess;
  a.part = part;
  a.status = status;
  a.spin_limit = spin_limit;
  static int granted[64] = {};
  const cudaError_t err = grant_smem(wide_gram_tc_kernel, kWtSmem, granted);
  if (err != cudaSuccess) return err;
  pdl_launch(wide_gram_tc_kernel, jobs, kWtThreads, kWtSmem, s, a);
  count_launches(1);
  return cudaGetLastError();
}

bool wide_tc_encode(const WideTcBlock& b, WideTcEntry* e) {
  std::memset(static_cast<void*>(e), 0, sizeof(*e));
  e->b = b;
  return b.part != nullptr && b.status != nullptr && encode_wt_map(&e->map, b);
}

bool wide_form_encode(const WideFormBlock& b, WideFormEntry* e) {
  std::memset(static_cast<void*>(e), 0, sizeof(*e));
  e->b = b;
  return b.status != nullptr && form_block_ok(b) && form_w_ok(b.WT, b.WTlo, b.n) &&
         encode_wf_map(&e->xmap, b.X, b.k, b.rows, b.ldx) && encode_wf_map(&e->wmap, b.WT, b.n, b.n, b.n) &&
         encode_wf_map(&e->wlmap, b.WTlo, b.n, b.n, b.n);
}

cudaError_t launch_wide_gram_tc_table(const WideTcEntry* e, const int32_t* job0, int nb, int ctas,
                                      int64_t spin_limit, cudaStream_t s) {
  if (nb <= 0 || ctas <= 0) return cudaSuccess;
  if ((reinterpret_cast<uintptr_t>(e) & 127) != 0) return cudaErrorInvalidValue;
  static int granted[64] = {};
  const cudaError_t err = grant_smem(wide_gram_tc_table_kernel, kWtSmem, granted);
  if (err != cudaSuccess) return err;
  pdl_launch(wide_gram_tc_table_kernel, ctas, kWtThreads, kWtSmem, s, e, job0, nb, spin_limit);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_wide_form_tc_table(const WideFormEntry* e, const int32_t* job0, int nb, int ctas,
                                      int64_t spin_limit, cudaStream_t s) {
  if (nb <= 0 || ctas <= 0) return cudaSuccess;
  if ((reinterpret_cast<uintptr_t>(e) & 127) != 0) return cudaErrorInvalidValue;
  static int granted[64] = {};
  const cudaError_t err = grant_smem(wide_form_tc_table_kernel, kWfSmem, granted);
  if (err != cudaSuccess) return err;
  pdl_launch(wide_form_tc_table_kernel, ctas, kWtThreads, kWfSmem, s, e, job0, nb, spin_limit);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_wide_prep_table(const WidePrepEntry* e, const int32_t* cta0, int nb, int ctas, cudaStream_t s) {
  if (nb <= 0 || ctas <= 0) return cudaSuccess;
  pdl_launch(wide_prep_table_kernel, ctas, 256, 0, s, e, cta0, nb);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_wide_form_prep(const float* W, int n, float* WT, float* WTlo, cudaStream_t s) {
  const int64_t ne = static_cast<int64_t>(n) * n;
  pdl_launch(wide_form_prep_kernel, static_cast<int>((ne + 255) / 256), 256, 0, s, W, n, WT, WTlo);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_wide_form_tc(const WideFormBlock b[3], const float* WT, const float* WTlo, int n, int32_t* status,
                                int64_t spin_limit, cudaStream_t s) {
  WideFormArgs a;
  std::memset(&a, 0, sizeof(a));
  if (!form_w_ok(WT, WTlo, n)) return cudaErrorInvalidValue;
  if (!encode_wf_map(&a.wmap, WT, n, n, n) || !encode_wf_map(&a.wlmap, WTlo, n, n, n)) return cudaErrorInvalidValue;
  int jobs = 0;
  for (int i = 0; i < 3; ++i) {
    a.b[i] = b[i];
    a.job0[i] = jobs;
    jobs += b[i].njobs;
    if (b[i].njobs == 0) continue;
    if (!form_block_ok(b[i])) return cudaErrorInvalidValue;
    if (!encode_wf_map(&a.xmap[i], b[i].X, b[i].k, b[i].rows, b[i].ldx)) return cudaErrorInvalidValue;
  }
  if (jobs == 0) return cudaSuccess;
  a.status = status;
  a.spin_limit = spin_limit;
  static int granted[64] = {};
  const cudaError_t err = grant_smem(wide_form_tc_kernel, kWfSmem, granted);
  if (err != cudaSuccess) return err;
  pdl_launch(wide_form_tc_kernel, jobs, kWtThreads, kWfSmem, s, a);
  count_launches(1);
  return cudaGetLastError();
}

bool gram_tc_supported(int k, int kout) { return k % 4 == 0 && k <= 64 && kout <= 64 && encoder() != nullptr; }

cudaError_t launch_gram_tc_block(const void* X, int k, int64_t rows, const int64_t* rows_dev, const float* W, int wld,
                                 int kout, double* part, int grid_max, int num_sms, int* grid_used, int32_t* status,
                                 int64_t spin_limit, int withhold, cudaStream_t s, const void* X1, int k1,
                                 int64_t rows1) {
  const int kk = W ? kout : k;
  if (X1 && !(W && k1 >= 1 && k1 <= k && gram_tc_packs(k, kout, true))) return cudaErrorInvalidValue;
  if (gram_tc_packs(k, kout, W != nullptr)) {  // packed-operand engine: persistent CTAs, one per SM
    const int rr = 64 / kk;
    const int64_t tile_rows = W ? kTileRows : static_cast<int64_t>(kTileRows) * rr;
    int grid = static_cast<int>((rows + tile_rows - 1) / tile_rows + (X1 ? (rows1 + tile_rows - 1) / tile_rows : 0));
    if (grid > num_sms) grid = num_sms;
    if (grid > grid_max) grid = grid_max;
    if (grid < 1) grid = 1;
    *grid_used = grid;
    PackArgs a{};
    a.k = k;
    a.kout = kout;
    a.np = (kout + 15) / 16 * 16;
    a.ksteps_f = (k + 7) / 8;
    a.kk = kk;
    a.rr = rr;
    a.rows = rows;
    a.rows_dev = rows_dev;
    a.W = W;
    a.wld = wld;
    a.part = part;
    a.status = status;
    a.spin_limit = spin_limit;
    a.withhold = withhold;
    a.rows1 = X1 ? rows1 : 0;
    CUtensorMap map, map1;
    cuuint32_t box[2] = {32, static_cast<cuuint32_t>(kTileRows)};
    cuuint32_t es[2] = {1, 1};
    CUresult cr;
    // rows of X (k columns; the 32-column box reads zeros past them), K-major operand of the formation product
    auto x_map = [&](CUtensorMap* m, const void* Xp, int kc, int64_t nr) {
      cuuint64_t dims[2] = {static_cast<cuuint64_t>(kc), static_cast<cuuint64_t>(nr > 0 ? nr : 1)};
      cuuint64_t strides[1] = {static_cast<cuuint64_t>(kc) * 4};
      return encoder()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(Xp), dims, strides, box, es,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    };
    if (W) {
      cr = x_map(&map, X, k, rows);
      if (cr == CUDA_SUCCESS) cr = X1 ? x_map(&map1, X1, k1, rows1) : CUDA_SUCCESS;
      if (!X1) map1 = map;
    } else {  // packed rows: rr consecutive rows = one 64-column row (the last one may run into the next array)
      const int64_t wrows = (rows + rr - 1) / rr;
      cuuint64_t dims[2] = {64, static_cast<cuuint64_t>(wrows > 0 ? wrows : 1)};
      cuuint64_t strides[1] = {256};
      cr = encoder()(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(X), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B_ATOM_32B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      map1 = map;
    }
    if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;
    static int granted[64][8] = {};
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    const int which = (kk == 4 ? 0 : (kk == 8 ? 1 : (kk == 16 ? 2 : 3))) + (W ? 4 : 0);
    void (*const kerns[8])(const CUtensorMap, const CUtensorMap, PackArgs) = {
        gram_pack_kernel<4, false>, gram_pack_kernel<8, false>, gram_pack_kernel<16, false>, gram_pack_kernel<32, false>,
        gram_pack_kernel<4, true>,  gram_pack_kernel<8, true>,  gram_pack_kernel<16, true>,  gram_pack_kernel<32, true>};
    void (*kern)(const CUtensorMap, const CUtensorMap, PackArgs) = kerns[which];
    if (dev < 0 || dev >= 64 || !granted[dev][which]) {
      err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kPackSmemBytes);
      if (err != cudaSuccess) return err;
      if (dev >= 0 && dev < 64) granted[dev][which] = 1;
    }
    pdl_launch(kern, grid, kPackThreads, kPackSmemBytes, s, map, map1, a);
    count_launches(1);
    return cudaGetLastError();
  }
  if (k <= 32 && kout <= 32) {  // pipelined engine: persistent CTAs, one per SM
    int grid = static_cast<int>((rows + kTileRows - 1) / kTileRows);
    if (grid > num_sms) grid = num_sms;
    if (grid > grid_max) grid = grid_max;
    if (grid < 1) grid = 1;
    *grid_used = grid;
    PipeArgs a{};
    a.k = k;
    a.kout = kout;
    a.np = (kout + 15) / 16 * 16;
    a.ksteps_f = (k + 7) / 8;
    a.rows = rows;
    a.rows_dev = rows_dev;
    a.W = W;
    a.wld = wld;
    a.part = part;
    a.status = status;
    a.spin_limit = spin_limit;
    CUtensorMap map;
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(k), static_cast<cuuint64_t>(rows > 0 ? rows : 1)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(k) * 4};
    cuuint32_t box[2] = {32, static_cast<cuuint32_t>(kTileRows)};
    cuuint32_t es[2] = {1, 1};
    const CUtensorMapSwizzle sw = W ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_128B_ATOM_32B;
    CUresult cr = encoder()(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(X), dims, strides, box, es,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;
    static int granted[64] = {0};
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (dev < 0 || dev >= 64 || !granted[dev]) {
      err = cudaFuncSetAttribute(gram_pipe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kPipeSmemBytes);
      if (err != cudaSuccess) return err;
      if (dev >= 0 && dev < 64) granted[dev] = 1;
    }
    pdl_launch(gram_pipe_kernel, grid, kPipeThreads, kPipeSmemBytes, s, map, a);
    count_launches(1);
    return cudaGetLastError();
  }
  const int grid = grid_max;
  *grid_used = grid;
  Geometry g = geometry(k, kout, W != nullptr);
  TcArgs a = g.a;
  a.rows = rows;
  a.rows_dev = rows_dev;
  a.W = W;
  a.wld = wld;
  a.part = part;
  a.status = status;
  a.spin_limit = spin_limit;
  CUtensorMap map;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(k), static_cast<cuuint64_t>(rows > 0 ? rows : 1)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(k) * 4};
  cuuint32_t box[2] = {32, static_cast<cuuint32_t>(kTileRows)};
  cuuint32_t es[2] = {1, 1};
  // pass 1 feeds the tile to the Gram as MN-major operands (32-byte atoms);
  // pass 2 feeds it to the formation product as the K-major operand
  const CUtensorMapSwizzle sw = W ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_128B_ATOM_32B;
  CUresult cr = encoder()(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(X), dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;
  cudaError_t err;
  if (a.np <= 32) {
    err = cudaFuncSetAttribute(gram_tc_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(g.smem));
    if (err != cudaSuccess) return err;
    pdl_launch(gram_tc_kernel<32>, grid, kTcThreads, g.smem, s, map, a);
  } else {
    err = cudaFuncSetAttribute(gram_tc_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(g.smem));
    if (err != cudaSuccess) return err;
    pdl_launch(gram_tc_kernel<64>, grid, kTcThreads, g.smem, s, map, a);
  }
  count_launches(1);
  return cudaGetLastError();
}

// Batched tensor-core Gram.  Engine of Gram block b in a pass: 0 = none (the
// CUDA-core engine takes it), 1 = packed (variant 0..3 for widths 4, 8, 16,
// 32), 2 = general (variant 0, 1 for N = 32, 64); with its tile rows and
// shared memory.
int gram_tc_batch_engine(const Plan& p, int pass, int b, int* variant, int64_t* tile_rows, size_t* smem) {
  if (!p.mixed || p.gram_engine == 1) return 0;
  const BlockShape sh = block_shape(p, pass, b);
  if (sh.rows == 0 || !gram_tc_supported(sh.k, sh.kout)) return 0;
  if (gram_tc_packs(sh.k, sh.kout, pass == 2)) {
    const int kk = pass == 2 ? sh.kout : sh.k;
    *variant = kk == 4 ? 0 : (kk == 8 ? 1 : (kk == 16 ? 2 : 3));
    *tile_rows = pass == 2 ? kTileRows : static_cast<int64_t>(kTileRows) * (64 / kk);
    *smem = kPackSmemBytes;
    return 1;
  }
  const Geometry g = geometry(sh.k, sh.kout, pass == 2);
  *variant = g.a.np <= 32 ? 0 : 1;
  *tile_rows = kTileRows;
  *smem = g.smem;
  return 2;
}

namespace {

// The tensor map of a batched job, encoded as the single-instance launcher does.
bool batch_map(const Plan& p, int pass, int b, int engine, CUtensorMap* map) {
  const BlockShape sh = block_shape(p, pass, b);
  cuuint32_t box[2] = {32, static_cast<cuuint32_t>(kTileRows)};
  cuuint32_t es[2] = {1, 1};
  CUresult cr;
  if (engine == 1 && pass == 1) {  // packed rows of 64 values
    const int rr = 64 / sh.k;
    const int64_t wrows = (sh.rows + rr - 1) / rr;
    cuuint64_t dims[2] = {64, static_cast<cuuint64_t>(wrows > 0 ? wrows : 1)};
    cuuint64_t strides[1] = {256};
    cr = encoder()(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(sh.X), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B_ATOM_32B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else {
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(sh.k), static_cast<cuuint64_t>(sh.rows > 0 ? sh.rows : 1)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(sh.k) * 4};
    // the packed engine's pass 2 and the general engine's pass 2 read X as the
    // K-major operand of the formation product; the general engine's pass 1
    // as MN-major Gram operands (32-byte atoms)
    const CUtensorMapSwizzle sw =
        pass == 2 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_128B_ATOM_32B;
    cr = encoder()(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(sh.X), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  return cr == CUDA_SUCCESS;
}

}  // namespace

cudaError_t launch_gram_tc_batch(const Plan* dev_plans, const Plan* host_plans, int pass, int engine, int variant,
                                 const TcJob* jobs, int njobs, size_t smem, cudaStream_t s) {
  if (njobs == 0) return cudaSuccess;
  void (*kern)(const TcBatch) = nullptr;
  if (engine == 1) {
    void (*const kerns[8])(const TcBatch) = {gram_pack_batched<4, false>, gram_pack_batched<8, false>,
                                             gram_pack_batched<16, false>, gram_pack_batched<32, false>,
                                             gram_pack_batched<4, true>,  gram_pack_batched<8, true>,
                                             gram_pack_batched<16, true>, gram_pack_batched<32, true>};
    kern = kerns[(variant & 3) + (pass == 2 ? 4 : 0)];
  }
  else
    kern = variant == 0 ? gram_tc_batched<32> : gram_tc_batched<64>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  TcBatch B;
  std::memset(&B, 0, sizeof(B));
  for (int j0 = 0; j0 < njobs; j0 += kTcJobs) {
    const int nj = njobs - j0 < kTcJobs ? njobs - j0 : kTcJobs;
    B.plans = dev_plans;
    B.njobs = nj;
    B.pass = pass;
    B.first[0] = 0;
    for (int j = 0; j < nj; ++j) {
      const TcJob& J = jobs[j0 + j];
      if (!batch_map(host_plans[J.inst], pass, J.blk, engine, &B.maps[j])) return cudaErrorInvalidValue;
      B.inst[j] = J.inst;
      B.blk[j] = static_cast<int8_t>(J.blk);
      B.first[j + 1] = B.first[j] + J.ctas;
    }
    pdl_launch(kern, B.first[nj], engine == 1 ? kPackThreads : kTcThreads, smem, s, B);
    count_launches(1);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  return cudaSuccess;
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

}  // namespace figaro
