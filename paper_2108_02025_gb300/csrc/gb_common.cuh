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

// Correctly rounded fma in the element type.
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// Sum over aligned groups of W lanes with an xor butterfly: every lane of a
// group ends with the same, order-fixed total.
template <int W>
__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// c_i <- c_i + alpha * s, computed in FP64 and rounded once to T.
template <typename T>
__device__ __forceinline__ T update(T c0, T alpha, double s) {
  return (T)__fma_rn((double)alpha, s, (double)c0);
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

// Arrival counter of one output tile.  Called by every thread of a block
// after the block wrote its partial sums: returns true in the block that
// arrived last (which then owns the final, fixed-order reduction).  The
// fence/atomic pair publishes the partials of all earlier blocks to it.
__device__ __forceinline__ bool arrive_last(unsigned* ticket, unsigned expected, int* flag) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned prev = atomicAdd(ticket, 1u);
    *flag = (prev == expected - 1);
  }
  __syncthreads();
  const bool last = *flag != 0;
  if (last) __threadfence();
  return last;
}

// Sum `count` partial values per output row, value q of row r being
// src[q * stride + row0 + r], in index order q = 0, 1, ... (cut into slices
// so that all threads load at once; slices are combined in slice order
// through shared memory), then hand (row, sum) to `sink` once per row.
// `red` must hold kThreads doubles.  Synchronises the block.
template <typename Sink>
__device__ void sum_rows(const double* src, int64_t stride, int count, int64_t row0, int64_t rows,
                         double* red, Sink sink) {
  int nslice = kThreads / (int)(rows < kThreads ? rows : kThreads);
  if (nslice > count) nslice = count;
  const int per = (count + nslice - 1) / nslice;
  const int64_t crow = kThreads / nslice;  // rows handled per pass
  for (int64_t base = 0; base < rows; base += crow) {
    const int64_t r = base + threadIdx.x % crow;
    const int slice = (int)(threadIdx.x / crow);
    double s = 0.0;
    if (slice < nslice && r < rows) {
      const int q0 = slice * per;
      const int q1 = q0 + per < count ? q0 + per : count;
      const double* p = src + row0 + r;
      int q = q0;
      for (; q + 8 <= q1; q += 8) {  // eight loads in flight, added in order
        double v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = __ldcg(p + (int64_t)(q + k) * stride);
#pragma unroll
        for (int k = 0; k < 8; ++k) s = __dadd_rn(s, v[k]);
      }
      for (; q < q1; ++q) s = __dadd_rn(s, __ldcg(p + (int64_t)q * stride));
    }
    red[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x < crow && base + threadIdx.x < rows) {
      double t = 0.0;
      for (int k = 0; k < nslice; ++k) t = __dadd_rn(t, red[k * crow + threadIdx.x]);
      sink(row0 + base + threadIdx.x, t);
    }
    __syncthreads();
  }
}

// Called by every thread of the block that wrote partial `s` of the rows
// [row0, row0 + rows) of tile `tile`.  The last block of each group sums the
// group; the last group sums the groups and applies c <- c + alpha*sum.
// Every counter is back at zero when the call's last block finishes.
template <typename T>
__device__ void split_finish(const Split& sp, int64_t tile, int s, int64_t row0, int64_t rows,
                             T* c, T alpha, double* red, int* flag) {
  const int g = s / kGroup;
  const int gsize = (g + 1) * kGroup <= sp.S ? kGroup : sp.S - g * kGroup;
  unsigned* t1 = sp.tickets + tile * (sp.NG + 1) + g;
  unsigned* t2 = sp.tickets + tile * (sp.NG + 1) + sp.NG;
  if (!arrive_last(t1, (unsigned)gsize, flag)) return;
  const double* src = sp.part + (int64_t)g * kGroup * sp.m;
  if (sp.NG == 1) {
    sum_rows(src, sp.m, gsize, row0, rows, red,
             [&](int64_t row, double v) { c[row] = update(c[row], alpha, v); });
    if (threadIdx.x == 0) *t1 = 0u;
    return;
  }
  sum_rows(src, sp.m, gsize, row0, rows, red,
           [&](int64_t row, double v) { sp.part2[(int64_t)g * sp.m + row] = v; });
  if (threadIdx.x == 0) *t1 = 0u;
  if (!arrive_last(t2, (unsigned)sp.NG, flag)) return;
  sum_rows(sp.part2, sp.m, sp.NG, row0, rows, red,
           [&](int64_t row, double v) { c[row] = update(c[row], alpha, v); });
  if (threadIdx.x == 0) *t2 = 0u;
}

}  // namespace gb
