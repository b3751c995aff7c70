// Shared device helpers of the GEMV / DOT / GER kernels (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gb_internal.h"

namespace gb {

// V consecutive elements of T moved as one 16-byte access when V > 1.
template <typename T, int V>
struct Pack {
  T v[V];
};

// Read-once data (A, the DOT vectors, C of GER): streaming load, evict first.
template <typename T, int V>
__device__ __forceinline__ Pack<T, V> ld_stream(const T* p) {
  Pack<T, V> r;
  if constexpr (V == 1) {
    r.v[0] = __ldcs(p);
  } else if constexpr (sizeof(T) == 4 && V == 4) {
    float4 q = __ldcs(reinterpret_cast<const float4*>(p));
    r.v[0] = q.x; r.v[1] = q.y; r.v[2] = q.z; r.v[3] = q.w;
  } else {
    static_assert(sizeof(T) == 8 && V == 2, "16-byte packs only");
    double2 q = __ldcs(reinterpret_cast<const double2*>(p));
    r.v[0] = q.x; r.v[1] = q.y;
  }
  return r;
}

// Reused data (x of GEMV, the vectors of GER): read-only path, cached.
template <typename T, int V>
__device__ __forceinline__ Pack<T, V> ld_keep(const T* p) {
  Pack<T, V> r;
  if constexpr (V == 1) {
    r.v[0] = __ldg(p);
  } else if constexpr (sizeof(T) == 4 && V == 4) {
    float4 q = __ldg(reinterpret_cast<const float4*>(p));
    r.v[0] = q.x; r.v[1] = q.y; r.v[2] = q.z; r.v[3] = q.w;
  } else {
    static_assert(sizeof(T) == 8 && V == 2, "16-byte packs only");
    double2 q = __ldg(reinterpret_cast<const double2*>(p));
    r.v[0] = q.x; r.v[1] = q.y;
  }
  return r;
}

template <typename T, int V>
__device__ __forceinline__ void st_stream(T* p, const Pack<T, V>& r) {
  if constexpr (V == 1) {
    __stcs(p, r.v[0]);
  } else if constexpr (sizeof(T) == 4 && V == 4) {
    __stcs(reinterpret_cast<float4*>(p), make_float4(r.v[0], r.v[1], r.v[2], r.v[3]));
  } else {
    __stcs(reinterpret_cast<double2*>(p), make_double2(r.v[0], r.v[1]));
  }
}

// ---- asynchronous global -> shared copies (cp.async), 16 bytes per lane.
// Each lane copies, waits for and reads back only its own slots, so no
// barrier is needed between lanes; the hardware tracks completion per thread.
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
// Streamed data: bypass L1 (.cg).
__device__ __forceinline__ void cp_async_cg16(unsigned dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
// Reused data (x): through L1 (.ca).
__device__ __forceinline__ void cp_async_ca16(unsigned dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_ca4(unsigned dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src) : "memory");
}
// One element (4 or 8 bytes) through L1, for a value read long before use.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_u32(dst)), "l"(src), "n"(sizeof(T))
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <typename T, int V>
__device__ __forceinline__ Pack<T, V> lds_pack(const unsigned char* p) {
  Pack<T, V> r;
  if constexpr (sizeof(T) == 4 && V == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    r.v[0] = q.x; r.v[1] = q.y; r.v[2] = q.z; r.v[3] = q.w;
  } else {
    static_assert(sizeof(T) == 8 && V == 2, "16-byte packs only");
    const double2 q = *reinterpret_cast<const double2*>(p);
    r.v[0] = q.x; r.v[1] = q.y;
  }
  return r;
}

// Correctly rounded fma in the element type.
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// ---- FP64 products on the FP32 pipe --------------------------------------
// GB300 issues FP64 FMAs at about 2 per clock per SM, too few for an FP64
// GEMV to keep up with HBM.  The FP64 GEMV kernels therefore form part of
// their products a*x with FP32 instructions: each operand is cut into a
// 24-bit head and the next 23 bits (emu_split, integer operations on the
// bit pattern, exact), the head product is formed exactly with an FMA
// (TwoProduct), the two cross terms are added in FP32, and the running sum
// is an unevaluated FP32 pair (H, L) updated with Knuth's TwoSum.  The
// operand cuts drop below 3*2^-46 of |a*x| per product and the rounding of
// the cross terms below 2^-45; the pair is folded into the FP64 sum every
// kEmuChain products or fewer.  Operands outside 2^-30 <= |v| < 2^34 (zero,
// subnormal, huge, Inf, NaN) take the FP64 FMA instead (emu_ok).

// Range of the emulated operands: the biased FP64 exponent in [993, 1056],
// i.e. 2^-30 <= |v| < 2^34.  emu_range(v) is below kEmuRange exactly for
// those: a valid operand sets bits below bit 26 only, any other some bit at
// 26 or above, so OR-ing several operands' values and comparing once tests
// them all.
constexpr unsigned kEmuRange = 64u << 20;
__device__ __forceinline__ unsigned emu_range(double v) {
  return ((unsigned)__double2hiint(v) & 0x7FF00000u) - (993u << 20);
}
__device__ __forceinline__ bool emu_ok(double v) { return emu_range(v) < kEmuRange; }

// v == hi + lo + r with |r| < 2^-46 |v|: hi = v truncated to 24 significant
// bits, lo = the next 23 bits.  Requires emu_ok(v).  In that range the
// rebiased exponent fits 8 bits, so the funnel shift leaves bit 31 clear for
// the sign; lo is (its 23 bits with hi's sign and exponent - 23) minus the
// implicit leading one, an exact subtraction.
__device__ __forceinline__ void emu_split(double v, float& hi, float& lo) {
  const unsigned h = (unsigned)__double2hiint(v), l = (unsigned)__double2loint(v);
  const unsigned f = __funnelshift_l(l, h - (896u << 20), 3);  // rebias 1023 -> 127, shift into place
  const unsigned hb = f | (h & 0x80000000u);
  hi = __uint_as_float(hb);
  const unsigned sg = (hb & 0xFF800000u) - (23u << 23);        // sign, exponent 23 below hi's
  lo = __fsub_rn(__uint_as_float(sg | ((l >> 6) & 0x7FFFFFu)), __uint_as_float(sg));
}

// (H, L) += a*x with FP32 instructions only; requires emu_ok(a) && emu_ok(x).
__device__ __forceinline__ void emu_fma(float ah, float al, float xh, float xl, float& H, float& L) {
  const float p = __fmul_rn(ah, xh);
  const float e = __fmaf_rn(ah, xh, -p);              // ah*xh == p + e exactly
  const float t = __fmaf_rn(ah, xl, __fmaf_rn(al, xh, e));
  const float s = __fadd_rn(H, p);                    // TwoSum(H, p)
  const float z = __fsub_rn(s, H);
  const float err = __fadd_rn(__fsub_rn(H, __fsub_rn(s, z)), __fsub_rn(p, z));
  H = s;
  L = __fadd_rn(L, __fadd_rn(err, t));
}

// At most this many emulated products enter one FP32 pair before it is
// folded into an FP64 sum (emu_fold).  With K products per pair and S the
// sum of their |a x|, H + L differs from the sum of the products' p + t by
// at most u^2 (K(K+1)/2 + 6K + 5) S (u = 2^-24: the TwoSum errors are below
// u S each, L's two roundings per product below u|err + t| and u|L|); with
// the 2.5*2^-45 per product of the operand cuts and of t, a chain of 16 is
// within 9.2e-13 of S (a chain of 32 would be within 2.7e-12).
constexpr int kEmuChain = 16;

// FP64 value of an FP32 pair word by integer operations (no FP64
// instruction: the small FP64 pipe is the limit of the FP64 kernels); exact
// for zero and normal numbers.  A subnormal word (below 2^-126, reachable
// only by cancellation inside a cross term) is taken as zero: an error below
// 2^-126 beside a sum of |a x| of at least 2^-60 (both operands pass emu_ok).
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned sgn = b & 0x80000000u;
  const bool nz = (b & 0x7F800000u) != 0u;
  const unsigned hi = nz ? (((b & 0x7FFFFFFFu) >> 3) + (896u << 20)) | sgn : sgn;
  const unsigned lo = nz ? b << 29 : 0u;
  return __hiloint2double((int)hi, (int)lo);
}

// acc <- acc + (H + L) with two FP64 additions, the pair reset to zero.
__device__ __forceinline__ void emu_fold(double& acc, float& H, float& L) {
  acc = __dadd_rn(acc, __dadd_rn(f2d_exact(H), f2d_exact(L)));
  H = 0.f;
  L = 0.f;
}

// The FP64 fallback of a group of emulated packs (an operand out of range):
// kept out of line, so that the hot path holds no FP64 instruction even when
// the compiler predicates the branch around the call.
template <int NP>
struct DPacks {
  double a[NP], x[NP];
};
template <int NP>
__device__ __noinline__ double dfma_fallback(const DPacks<NP> p, double acc) {
#pragma unroll
  for (int k = 0; k < NP; ++k) acc = __fma_rn(p.a[k], p.x[k], acc);
  return acc;
}

// Sum over aligned groups of W lanes with an xor butterfly: every lane of a
// group ends with the same, order-fixed total.
template <int W>
__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// c_i <- c_i + alpha * s in the element type: one fma.  (FP32 paths avoid
// FP64 instructions altogether: on this GPU every FP64 warp instruction,
// even with one active lane, occupies the small FP64 pipe.)
__device__ __forceinline__ float update(float c0, float alpha, float s) { return __fmaf_rn(alpha, s, c0); }
__device__ __forceinline__ double update(double c0, double alpha, double s) { return __fma_rn(alpha, s, c0); }
// The same from an FP64 partial sum (split sums are combined in FP64).
__device__ __forceinline__ float update_from(float c0, float alpha, double s) { return __fmaf_rn(alpha, (float)s, c0); }
__device__ __forceinline__ double update_from(double c0, double alpha, double s) { return __fma_rn(alpha, s, c0); }

// Error-free sum of two floats (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// Block-wide sum of one double per thread, in a fixed order (warp butterfly,
// then warps 0..7 in order).  Result valid in thread 0.  Uses `red` (8
// doubles of shared memory) and synchronises the block.
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = group_sum<32>(v);
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) t = __dadd_rn(t, red[w]);
  }
  __syncthreads();
  return t;
}

// Release/acquire fence at GPU scope.
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// Counter increment with release and acquire semantics at GPU scope, one
// instruction: the writes ordered before it (the caller's, and through a
// barrier those of its block) are published with it, and the reads ordered
// after it see what earlier arrivals published.  Returns the old value.
__device__ __forceinline__ unsigned arrive_add(unsigned* ticket) {
  unsigned prev;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(prev) : "l"(ticket) : "memory");
  return prev;
}

// Arrival counter of one output tile.  Called by every thread of a block
// after the block wrote its partial sums: returns true in the block that
// arrived last (which then owns the final, fixed-order reduction).  The
// barrier orders the block's partials before thread 0's counter increment
// (release); in the last block the second barrier orders every thread's
// reads of the other blocks' partials after it (acquire).  One thread
// synchronises with the other blocks instead of every thread of the block.
__device__ __forceinline__ bool arrive_last(unsigned* ticket, unsigned expected, int* flag) {
  __syncthreads();
  if (threadIdx.x == 0) *flag = arrive_add(ticket) == expected - 1;
  __syncthreads();
  return *flag != 0;
}

// Sum over aligned groups of W lanes in the element type (FP32 partials
// stay on the FP32 pipe), same fixed butterfly order as group_sum.
template <int W>
__device__ __forceinline__ float group_sum_f(float v) {
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Arrival counter of one output tile, for a warp that has written its
// partial sums (every lane that wrote calls this with the whole warp).
// Returns true in the warp that arrived last; the fence/atomic pair makes
// the partials of every earlier warp visible to it.
__device__ __forceinline__ bool warp_arrive_last(unsigned* ticket, unsigned expected) {
  __syncwarp();  // orders the warp's partials before lane 0's increment (release)
  unsigned prev = 0;
  if ((threadIdx.x & 31) == 0) prev = arrive_add(ticket);
  prev = __shfl_sync(0xffffffffu, prev, 0);
  __syncwarp();  // and the warp's later reads after it (acquire)
  return prev == expected - 1;
}

// Warp-wide sum, for each of `rows` outputs, of `count` partials: value q
// of row r is src[q * stride + row0 + r].  The warp works on up to 32/P rows
// at once with P lanes per row; lane k of a row adds q = k, k+P, ... in
// order, and the P lanes are combined by the fixed butterfly.  `sink(row, v)`
// runs in the first lane of each row's group.
template <int P, typename Sink>
__device__ __forceinline__ void warp_sum_rows_p(const double* src, int64_t stride, int count,
                                                int64_t row0, int rows, Sink& sink) {
  const int lane = threadIdx.x & 31;
  const int k = lane % P;
  for (int rb = 0; rb < rows; rb += 32 / P) {
    const int r = rb + lane / P;
    double s = 0.0;
    if (r < rows)
      for (int q = k; q < count; q += 4 * P) {  // four loads in flight, added in index order
        double v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = q + i * P < count ? __ldcg(src + (int64_t)(q + i * P) * stride + row0 + r) : 0.0;
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (q + i * P < count) s = __dadd_rn(s, v[i]);
      }
    s = group_sum<P>(s);
    if (k == 0 && r < rows) sink(row0 + r, s);
  }
}

template <typename Sink>
__device__ __forceinline__ void warp_sum_rows(const double* src, int64_t stride, int count,
                                              int64_t row0, int rows, Sink sink) {
  // lanes per row: as many as fit when all rows are handled in one pass
  const int per = rows >= 32 ? 1 : 32 / rows;
  if (per >= 32) warp_sum_rows_p<32>(src, stride, count, row0, rows, sink);
  else if (per >= 16) warp_sum_rows_p<16>(src, stride, count, row0, rows, sink);
  else if (per >= 8) warp_sum_rows_p<8>(src, stride, count, row0, rows, sink);
  else if (per >= 4) warp_sum_rows_p<4>(src, stride, count, row0, rows, sink);
  else if (per >= 2) warp_sum_rows_p<2>(src, stride, count, row0, rows, sink);
  else warp_sum_rows_p<1>(src, stride, count, row0, rows, sink);
}

constexpr int kSumBatch = 8;  // partial loads in flight per thread, block_sum_rows

// Block-wide sum, for each of `rows` outputs, of `count` partials: value q
// of row r is src[q * stride + row0 + r].  The 256 threads are cut into
// slices of the partials so that all of them load at once: slice k adds its
// partials in index order, the slices are added in slice order through
// shared memory, and `sink(row, v)` runs once per row.  `red` holds 256
// doubles.  Synchronises the block.
template <typename Sink>
__device__ void block_sum_rows(const double* src, int64_t stride, int count, int64_t row0,
                               int64_t rows, double* red, Sink sink) {
  int nslice = kThreads / (int)(rows < kThreads ? rows : kThreads);
  if (nslice > count) nslice = count;
  const int per = (count + nslice - 1) / nslice;
  const int64_t crow = kThreads / nslice;  // rows per pass
  for (int64_t base = 0; base < rows; base += crow) {
    const int64_t r = base + threadIdx.x % crow;
    const int slice = (int)(threadIdx.x / crow);
    double acc = 0.0;
    if (slice < nslice && r < rows) {
      const int q0 = slice * per;
      const int q1 = q0 + per < count ? q0 + per : count;
      const double* p = src + row0 + r;
      // up to kSumBatch loads in flight (the last batch predicated), then
      // added in index order: one L2 round trip per kSumBatch partials
      for (int q = q0; q < q1; q += kSumBatch) {
        double v[kSumBatch];
#pragma unroll
        for (int k = 0; k < kSumBatch; ++k) v[k] = q + k < q1 ? __ldcg(p + (int64_t)(q + k) * stride) : 0.0;
#pragma unroll
        for (int k = 0; k < kSumBatch; ++k)
          if (q + k < q1) acc = __dadd_rn(acc, v[k]);
      }
    }
    __syncthreads();
    red[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < crow && base + threadIdx.x < rows) {
      double t = 0.0;
      for (int k = 0; k < nslice; ++k) t = __dadd_rn(t, red[k * crow + threadIdx.x]);
      sink(row0 + base + threadIdx.x, t);
    }
  }
  __syncthreads();
}

// Final step of a split sum for a block that has written partial `s` of the
// rows [row0, row0 + rows) of tile `tile` (called by every thread).  The
// last block of each group of sp.G splits sums the group, the last group
// sums the groups and applies c <- c + alpha*sum; counters return to zero.
template <typename T>
__device__ __noinline__ void block_split_finish(const Split& sp, int64_t tile, int s, int64_t row0,
                                                int64_t rows, T* c, T alpha, double* red, int* flag) {
  const int g = s / sp.G;
  const int gsize = (g + 1) * sp.G <= sp.S ? sp.G : sp.S - g * sp.G;
  unsigned* t1 = sp.tickets + tile * (sp.NG + 1) + g;
  unsigned* t2 = sp.tickets + tile * (sp.NG + 1) + sp.NG;
  if (!arrive_last(t1, (unsigned)gsize, flag)) return;
  const double* src = sp.part + (int64_t)g * sp.G * sp.m;
  if (sp.NG == 1) {
    block_sum_rows(src, sp.m, gsize, row0, rows, red,
                   [&](int64_t row, double v) { c[row] = update_from(c[row], alpha, v); });
    if (threadIdx.x == 0) *t1 = 0u;
    return;
  }
  block_sum_rows(src, sp.m, gsize, row0, rows, red,
                 [&](int64_t row, double v) { sp.part2[(int64_t)g * sp.m + row] = v; });
  if (threadIdx.x == 0) *t1 = 0u;
  if (!arrive_last(t2, (unsigned)sp.NG, flag)) return;
  block_sum_rows(sp.part2, sp.m, sp.NG, row0, rows, red,
                 [&](int64_t row, double v) { c[row] = update_from(c[row], alpha, v); });
  if (threadIdx.x == 0) *t2 = 0u;
}

// Final step of a split sum, run by the warp that wrote partial `s` of rows
// [row0, row0 + rows) of row item `item`.  The S partials of a row are
// combined in groups of sp.G consecutive splits by the last warp to arrive
// in each group, then across the NG groups by the last group; each sum is in
// index order, and every counter is back at zero when the call's last warp
// finishes.  Workspace layout: see gb_split.h.
template <typename T>
__device__ __noinline__ void warp_split_finish(const Split& sp, int64_t item, int s, int64_t row0, int rows,
                                  T* c, T alpha) {
  const int g = s / sp.G;
  const int gsize = (g + 1) * sp.G <= sp.S ? sp.G : sp.S - g * sp.G;
  unsigned* t1 = sp.tickets + item * (sp.NG + 1) + g;
  unsigned* t2 = sp.tickets + item * (sp.NG + 1) + sp.NG;
  if (!warp_arrive_last(t1, (unsigned)gsize)) return;
  const double* src = sp.part + (int64_t)g * sp.G * sp.m;
  const bool lane0 = (threadIdx.x & 31) == 0;
  if (sp.NG == 1) {
    warp_sum_rows(src, sp.m, gsize, row0, rows,
                  [&](int64_t row, double v) { c[row] = update_from(c[row], alpha, v); });
    if (lane0) *t1 = 0u;
    return;
  }
  warp_sum_rows(src, sp.m, gsize, row0, rows,
                [&](int64_t row, double v) { sp.part2[(int64_t)g * sp.m + row] = v; });
  if (lane0) *t1 = 0u;
  if (!warp_arrive_last(t2, (unsigned)sp.NG)) return;
  warp_sum_rows(sp.part2, sp.m, sp.NG, row0, rows,
                [&](int64_t row, double v) { c[row] = update_from(c[row], alpha, v); });
  if (lane0) *t2 = 0u;
}

}  // namespace gb
