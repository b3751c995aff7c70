// DOT, alpha <- alpha + sum_p x_p y_p.
//
// Alg. 3 of the paper (Sec. 4.3) is one micro-kernel call over the whole
// range for small n; Alg. 4 blocks the range by n_c, lets the blocks run in
// parallel and adds their sums into alpha.  Here block b of a one-wave grid
// owns the contiguous range [b*chunk, (b+1)*chunk) and streams x and y with
// 16-byte loads; with one block (small n, Alg. 3) it adds its total to
// alpha directly, otherwise the block that finishes last sums the block
// totals in index order in FP64 and adds them to alpha.
//
// FP64 inputs: half of each thread's products are FP64 fmas (four chains),
// the other half are formed with FP32 instructions (exact operand cuts,
// TwoProduct, TwoSum; gb_common.cuh) when every active lane has them in
// range, so the small FP64 pipe does not cap the HBM stream.  FP32 inputs use the compensated
// dot product Dot2 of Ogita, Rump & Oishi ("Accurate sum and dot product",
// SIAM J. Sci. Comput. 26(6), 2005: TwoProduct by fma, TwoSum by Knuth) in
// FP32 per thread, so no FP64 operation is spent per element, and move to
// FP64 for the block and final sums.
#include "gb_common.cuh"
#include "gb_internal.h"

namespace gb {
namespace {

constexpr int kDotEmu64 = 2;  // FP64: packs per step (of 4) formed on the FP32 pipe
// steps per FP32 pair: kDotEmu64 packs of 2 products each, at most kEmuChain products
constexpr int kDotEmuFlush = kDotEmu64 > 0 && kEmuChain / (2 * kDotEmu64) > 0 ? kEmuChain / (2 * kDotEmu64) : 1;

// Per-thread accumulator of the sum of products.
template <typename T>
struct DotAcc;

template <>
struct DotAcc<double> {
  // four independent chains: the FP64 fma's latency is long on GB300
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  __device__ __forceinline__ void add(double x, double y, int k) {
    switch (k & 3) {
      case 0: a0 = __fma_rn(x, y, a0); break;
      case 1: a1 = __fma_rn(x, y, a1); break;
      case 2: a2 = __fma_rn(x, y, a2); break;
      default: a3 = __fma_rn(x, y, a3); break;
    }
  }
  __device__ __forceinline__ double total() const { return __dadd_rn(__dadd_rn(a0, a1), __dadd_rn(a2, a3)); }
};

// Two independent Dot2 chains (p: running sum, s: running error).
template <>
struct DotAcc<float> {
  float p0 = 0.f, s0 = 0.f, p1 = 0.f, s1 = 0.f;
  __device__ __forceinline__ static void step(float x, float y, float& p, float& s) {
    const float h = __fmul_rn(x, y);
    const float r = __fmaf_rn(x, y, -h);     // h + r == x*y exactly
    const float t = __fadd_rn(p, h);         // TwoSum(p, h) = (t, q)
    const float z = __fsub_rn(t, p);
    const float q = __fadd_rn(__fsub_rn(p, __fsub_rn(t, z)), __fsub_rn(h, z));
    p = t;
    s = __fadd_rn(s, __fadd_rn(q, r));
  }
  __device__ __forceinline__ void add(float x, float y, int k) {
    if (k & 1) step(x, y, p1, s1);
    else step(x, y, p0, s0);
  }
  __device__ __forceinline__ double total() const {
    return __dadd_rn(__dadd_rn((double)p0, (double)s0), __dadd_rn((double)p1, (double)s1));
  }
};

template <typename T, int V, int U>
__global__ void __launch_bounds__(kThreads, 4)
    dot_kernel(int64_t n, const T* __restrict__ x, const T* __restrict__ y, T* __restrict__ alpha,
               int64_t chunk, double* __restrict__ part, unsigned* __restrict__ ticket) {
  __shared__ double red[kThreads];
  __shared__ int flag;

  const int64_t lo = (int64_t)blockIdx.x * chunk;
  const int64_t hi = (lo + chunk < n) ? lo + chunk : n;
  const int64_t hv = lo + ((hi - lo) / V) * V;  // end of whole packs
  constexpr int64_t STEP = (int64_t)kThreads * V;

  DotAcc<T> acc;
  float eh = 0.f, el = 0.f;  // FP64: the pair of the FP32-emulated products
  int ebody = 0;
  int64_t i = lo + (int64_t)threadIdx.x * V;
  for (; i + (U - 1) * STEP < hv; i += U * STEP) {
    Pack<T, V> xp[U], yp[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      xp[q] = ld_stream<T, V>(x + i + q * STEP);
      yp[q] = ld_stream<T, V>(y + i + q * STEP);
    }
    if constexpr (sizeof(T) == 8 && V == 2 && kDotEmu64 > 0) {
      // FP64: the last kDotEmu64 packs with FP32 instructions (emu_fma) when
      // every active lane has them in range, relieving the FP64 pipe
      constexpr int QE = U - kDotEmu64;
#pragma unroll
      for (int q = 0; q < QE; ++q)
#pragma unroll
        for (int v = 0; v < V; ++v) acc.add(xp[q].v[v], yp[q].v[v], q * V + v);
      unsigned rb = 0u;  // the emulated operands' ranges, OR-ed
#pragma unroll
      for (int q = QE; q < U; ++q)
#pragma unroll
        for (int v = 0; v < V; ++v) rb |= emu_range(xp[q].v[v]) | emu_range(yp[q].v[v]);
      if (__all_sync(__activemask(), rb < kEmuRange)) {
#pragma unroll
        for (int q = QE; q < U; ++q)
#pragma unroll
          for (int v = 0; v < V; ++v) {
            float xh, xl, yh, yl;
            emu_split(xp[q].v[v], xh, xl);
            emu_split(yp[q].v[v], yh, yl);
            emu_fma(xh, xl, yh, yl, eh, el);
          }
        if (++ebody == kDotEmuFlush) {
          ebody = 0;
          emu_fold(acc.a3, eh, el);
        }
      } else {
        DPacks<kDotEmu64 * V> dp;
#pragma unroll
        for (int q = QE; q < U; ++q)
#pragma unroll
          for (int v = 0; v < V; ++v) {
            dp.a[(q - QE) * V + v] = xp[q].v[v];
            dp.x[(q - QE) * V + v] = yp[q].v[v];
          }
        acc.a2 = dfma_fallback(dp, acc.a2);
      }
    } else {
#pragma unroll
      for (int q = 0; q < U; ++q)
#pragma unroll
        for (int v = 0; v < V; ++v) acc.add(xp[q].v[v], yp[q].v[v], q * V + v);
    }
  }
  for (; i < hv; i += STEP) {
    const Pack<T, V> xp = ld_stream<T, V>(x + i), yp = ld_stream<T, V>(y + i);
#pragma unroll
    for (int v = 0; v < V; ++v) acc.add(xp.v[v], yp.v[v], v);
  }
  for (int64_t k = hv + threadIdx.x; k < hi; k += kThreads) acc.add(__ldcs(x + k), __ldcs(y + k), 0);

  if constexpr (sizeof(T) == 8) emu_fold(acc.a3, eh, el);
  const double bsum = block_sum(acc.total(), red);

  if (gridDim.x == 1) {  // one block: Alg. 3, no workspace
    if (threadIdx.x == 0) *alpha = (T)__dadd_rn((double)*alpha, bsum);
    return;
  }
  if (threadIdx.x == 0) part[blockIdx.x] = bsum;
  if (arrive_last(ticket, gridDim.x, &flag)) {
    double s = 0.0;  // block totals, in index order per thread, then block_sum's fixed order
    const int per = (gridDim.x + kThreads - 1) / kThreads;
    const int b0 = threadIdx.x * per;
    for (int b = b0; b < b0 + per; b += 4) {  // four loads in flight, added in index order
      double v[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) v[i] = b + i < b0 + per && b + i < (int)gridDim.x ? __ldcg(part + b + i) : 0.0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (b + i < b0 + per && b + i < (int)gridDim.x) s = __dadd_rn(s, v[i]);
    }
    const double total = block_sum(s, red);
    if (threadIdx.x == 0) {
      *alpha = (T)__dadd_rn((double)*alpha, total);
      *ticket = 0u;
    }
  }
}

template <typename T, int V>
int launch(const DotArgs<T>& a, const DotPlan& p, cudaStream_t st) {
  dot_kernel<T, V, 4><<<(unsigned)p.blocks, kThreads, 0, st>>>(a.n, a.x, a.y, a.alpha, p.chunk,
                                                                p.part, p.ticket);
  return 0;
}

}  // namespace

template <typename T>
int dot_launch(const DotArgs<T>& a, const DotPlan& p, cudaStream_t st) {
  if (p.vec) return launch<T, 16 / sizeof(T)>(a, p, st);
  return launch<T, 1>(a, p, st);
}

template int dot_launch<float>(const DotArgs<float>&, const DotPlan&, cudaStream_t);
template int dot_launch<double>(const DotArgs<double>&, const DotPlan&, cudaStream_t);

}  // namespace gb
