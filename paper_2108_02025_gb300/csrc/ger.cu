// GER, C_ij <- fma(x_i, t_j, C_ij) with t_j = fl(alpha * y_j).
//
// Alg. 2 of the paper (Sec. 4.2): Loop-1 over the lines of C is the parallel
// loop; splitting Loop-2 among workers would race on C, so every element has
// exactly one writer here too.  A "line" is a row of a row-major C or a
// column of a column-major C.  One warp item is a segment of 32*V*U
// elements of a block of LB consecutive lines: the lane loads the
// along-line vector for its U packs once (t = alpha*y for rows, x for
// columns), then streams the LB lines past it, two at a time, with 16-byte
// streaming loads and stores, so alpha*y_j is formed once per LB lines
// rather than once per element.
#include "gb_common.cuh"
#include "gb_internal.h"

namespace gb {
namespace {

template <typename T, int V, int U, int LB, bool ROW>
__global__ void __launch_bounds__(kThreads)
    ger_kernel(int64_t lines, int64_t len, T alpha, const T* __restrict__ x,
               const T* __restrict__ y, T* __restrict__ C, int64_t ld, int64_t segs,
               int64_t items) {
  constexpr int64_t SEG = 32LL * V * U;
  const T* vsrc = ROW ? y : x;  // vector along a line
  const T* ssrc = ROW ? x : y;  // one scalar per line
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (kThreads / 32);

  for (int64_t w = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5; w < items; w += nwarps) {
    const int64_t lb = w / segs;
    const int64_t seg = w - lb * segs;
    const int64_t kb = seg * SEG + (int64_t)lane * V;

    Pack<T, V> vv[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int64_t k = kb + (int64_t)q * 32 * V;
      if (k + V <= len) {
        vv[q] = ld_keep<T, V>(vsrc + k);
      } else {
#pragma unroll
        for (int v = 0; v < V; ++v) vv[q].v[v] = (k + v < len) ? __ldg(vsrc + k + v) : T(0);
      }
      if constexpr (ROW) {
#pragma unroll
        for (int v = 0; v < V; ++v) vv[q].v[v] = mul_rn(alpha, vv[q].v[v]);
      }
    }

    const int64_t L0 = lb * LB;
    const int64_t L1 = (L0 + LB < lines) ? L0 + LB : lines;
    for (int64_t L = L0; L < L1; L += 2) {
      const bool two = L + 1 < L1;
      T s0 = __ldg(ssrc + L);
      T s1 = two ? __ldg(ssrc + L + 1) : T(0);
      if constexpr (!ROW) { s0 = mul_rn(alpha, s0); s1 = mul_rn(alpha, s1); }
      T* C0 = C + L * ld;
      T* C1 = C0 + ld;
      Pack<T, V> c0[U], c1[U];
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const int64_t k = kb + (int64_t)q * 32 * V;
        if (k + V <= len) {
          c0[q] = ld_stream<T, V>(C0 + k);
          if (two) c1[q] = ld_stream<T, V>(C1 + k);
        }
      }
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const int64_t k = kb + (int64_t)q * 32 * V;
        if (k + V <= len) {
#pragma unroll
          for (int v = 0; v < V; ++v)
            c0[q].v[v] = ROW ? fma_rn(s0, vv[q].v[v], c0[q].v[v]) : fma_rn(vv[q].v[v], s0, c0[q].v[v]);
          st_stream<T, V>(C0 + k, c0[q]);
          if (two) {
#pragma unroll
            for (int v = 0; v < V; ++v)
              c1[q].v[v] = ROW ? fma_rn(s1, vv[q].v[v], c1[q].v[v]) : fma_rn(vv[q].v[v], s1, c1[q].v[v]);
            st_stream<T, V>(C1 + k, c1[q]);
          }
        } else if (k < len) {  // ragged end of the line (< V elements)
          for (int v = 0; v < V && k + v < len; ++v) {
            C0[k + v] = ROW ? fma_rn(s0, vv[q].v[v], C0[k + v]) : fma_rn(vv[q].v[v], s0, C0[k + v]);
            if (two) C1[k + v] = ROW ? fma_rn(s1, vv[q].v[v], C1[k + v]) : fma_rn(vv[q].v[v], s1, C1[k + v]);
          }
        }
      }
    }
  }
}

template <typename T, int V, bool ROW>
int launch(const GerArgs<T>& a, const GerPlan& p, cudaStream_t st) {
  constexpr int U = 4, LB = 8;
  auto kern = ger_kernel<T, V, U, LB, ROW>;
  const int64_t segs = (p.len + 32LL * V * U - 1) / (32LL * V * U);
  const int64_t items = (p.lines + LB - 1) / LB * segs;
  const int64_t blocks = (items + kThreads / 32 - 1) / (kThreads / 32);
  const int grid = grid_size((const void*)kern, blocks);
  kern<<<grid, kThreads, 0, st>>>(p.lines, p.len, a.alpha, a.x, a.y, a.C, a.ldc, segs, items);
  return 0;
}

}  // namespace

template <typename T>
int ger_launch(const GerArgs<T>& a, const GerPlan& p, cudaStream_t st) {
  constexpr int V = 16 / sizeof(T);
  if (p.vec) return p.row ? launch<T, V, true>(a, p, st) : launch<T, V, false>(a, p, st);
  return p.row ? launch<T, 1, true>(a, p, st) : launch<T, 1, false>(a, p, st);
}

template int ger_launch<float>(const GerArgs<float>&, const GerPlan&, cudaStream_t);
template int ger_launch<double>(const GerArgs<double>&, const GerPlan&, cudaStream_t);

}  // namespace gb
