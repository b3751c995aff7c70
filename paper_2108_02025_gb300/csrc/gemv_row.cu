// Row-major GEMV, c_i <- c_i + alpha * sum_j A[i*lda + j] x_j.
//
// Alg. 2 of the paper (Sec. 4.2) hands each row, a unit-stride dot product,
// to one worker; Loop-1 (rows) is the parallel loop.  Here a row goes to a
// group of LPR lanes of a warp (LPR = 32 for long rows, fewer for short ones)
// that streams it with 16-byte loads; each group carries RW rows at once so
// that every x pack it loads serves RW rows and each lane has RW*U loads of
// A in flight.  When there are too few rows to fill the GPU, the columns are
// split into S chunks (the Alg. 4 idea of blocking the index range) and the
// chunk partials are summed in a fixed order by the block that finishes a
// row tile last.
#include "gb_common.cuh"
#include "gb_internal.h"

namespace gb {
namespace {

template <typename T, int V, int LPR, int RW, int U>
__global__ void __launch_bounds__(kThreads)
    gemv_row_kernel(int64_t m, int64_t n, T alpha, const T* __restrict__ A, int64_t lda,
                    const T* __restrict__ x, T* __restrict__ c, const Split sp, int64_t KC,
                    int64_t units) {
  const int S = sp.S;
  constexpr int GPW = 32 / LPR;                   // row groups per warp
  constexpr int GROUPS = kThreads / LPR;          // row groups per block
  constexpr int ROWS = GROUPS * RW;               // rows per block tile
  constexpr int64_t STEP = (int64_t)LPR * V;      // columns a group covers per pack
  // FP32 partial sums move into FP64 after at most 64 terms per lane
  constexpr int FLUSH = (sizeof(T) == 4) ? (64 / (U * V) > 0 ? 64 / (U * V) : 1) : 1 << 30;

  __shared__ double red[kThreads];
  __shared__ int flag;

  const int lane = threadIdx.x & 31;
  const int l = lane % LPR;
  const int grp = (threadIdx.x >> 5) * GPW + lane / LPR;

  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int64_t rt = u / S;
    const int s = (int)(u - rt * S);
    const int64_t row0 = rt * ROWS + (int64_t)grp * RW;
    const int64_t k0 = (int64_t)s * KC;
    const int64_t k1 = (k0 + KC < n) ? k0 + KC : n;
    const int64_t kv1 = k0 + ((k1 - k0) / V) * V;  // end of whole packs

    const T* Ar[RW];
#pragma unroll
    for (int r = 0; r < RW; ++r) {
      const int64_t row = (row0 + r < m) ? row0 + r : m - 1;  // clamp: the tail tile re-reads a row
      Ar[r] = A + row * lda;
    }

    double tot[RW];
    T acc[RW];
#pragma unroll
    for (int r = 0; r < RW; ++r) { tot[r] = 0.0; acc[r] = T(0); }

    int64_t j = k0 + (int64_t)l * V;
    int body = 0;
    for (; j + (U - 1) * STEP < kv1; j += U * STEP) {
      Pack<T, V> xp[U];
      Pack<T, V> ap[U][RW];
#pragma unroll
      for (int q = 0; q < U; ++q) {
        xp[q] = ld_keep<T, V>(x + j + q * STEP);
#pragma unroll
        for (int r = 0; r < RW; ++r) ap[q][r] = ld_stream<T, V>(Ar[r] + j + q * STEP);
      }
#pragma unroll
      for (int q = 0; q < U; ++q)
#pragma unroll
        for (int r = 0; r < RW; ++r)
#pragma unroll
          for (int v = 0; v < V; ++v) acc[r] = fma_rn(ap[q][r].v[v], xp[q].v[v], acc[r]);
      if constexpr (sizeof(T) == 4) {
        if (++body == FLUSH) {
          body = 0;
#pragma unroll
          for (int r = 0; r < RW; ++r) { tot[r] = __dadd_rn(tot[r], (double)acc[r]); acc[r] = 0.f; }
        }
      }
    }
    for (; j < kv1; j += STEP) {  // remaining whole packs
      const Pack<T, V> xq = ld_keep<T, V>(x + j);
#pragma unroll
      for (int r = 0; r < RW; ++r) {
        const Pack<T, V> aq = ld_stream<T, V>(Ar[r] + j);
#pragma unroll
        for (int v = 0; v < V; ++v) acc[r] = fma_rn(aq.v[v], xq.v[v], acc[r]);
      }
    }
    for (int64_t jj = kv1 + l; jj < k1; jj += LPR) {  // ragged end of the row (< V columns)
      const T xs = __ldg(x + jj);
#pragma unroll
      for (int r = 0; r < RW; ++r) acc[r] = fma_rn(__ldcs(Ar[r] + jj), xs, acc[r]);
    }

#pragma unroll
    for (int r = 0; r < RW; ++r) tot[r] = group_sum<LPR>(__dadd_rn(tot[r], (double)acc[r]));

    if (S == 1) {
      if (l == 0) {
#pragma unroll
        for (int r = 0; r < RW; ++r)
          if (row0 + r < m) c[row0 + r] = update(c[row0 + r], alpha, tot[r]);
      }
    } else {
      if (l == 0) {
#pragma unroll
        for (int r = 0; r < RW; ++r)
          if (row0 + r < m) sp.part[(int64_t)s * m + row0 + r] = tot[r];
      }
      const int64_t t0 = rt * ROWS;
      split_finish<T>(sp, rt, s, t0, (m - t0 < ROWS) ? m - t0 : ROWS, c, alpha, red, &flag);
    }
  }
}

template <typename T, int V, int LPR, int RW, int U>
int launch(const GemvArgs<T>& a, const GemvPlan& p, cudaStream_t st) {
  auto kern = gemv_row_kernel<T, V, LPR, RW, U>;
  const int grid = grid_size((const void*)kern, p.units);
  kern<<<grid, kThreads, 0, st>>>(a.m, a.n, a.alpha, a.A, a.lda, a.x, a.c, p.split, p.kc, p.units);
  return 0;
}

template <typename T, int V, int RW, int U>
int by_lpr(const GemvArgs<T>& a, const GemvPlan& p, cudaStream_t st) {
  switch (p.lpr) {
    case 32: return launch<T, V, 32, RW, U>(a, p, st);
    case 16: return launch<T, V, 16, RW, U>(a, p, st);
    case 8: return launch<T, V, 8, RW, U>(a, p, st);
    case 4: return launch<T, V, 4, RW, U>(a, p, st);
    case 2: return launch<T, V, 2, RW, U>(a, p, st);
    default: return launch<T, V, 1, RW, U>(a, p, st);
  }
}

}  // namespace

template <typename T>
int gemv_row_launch(const GemvArgs<T>& a, const GemvPlan& p, cudaStream_t st) {
  constexpr int V = 16 / sizeof(T);
  if (p.vec) {
    if (p.rw == 8) return by_lpr<T, V, 8, 2>(a, p, st);
    return by_lpr<T, V, 4, 2>(a, p, st);
  }
  if (p.rw == 8) return by_lpr<T, 1, 8, 2>(a, p, st);
  return by_lpr<T, 1, 4, 2>(a, p, st);
}

template int gemv_row_launch<float>(const GemvArgs<float>&, const GemvPlan&, cudaStream_t);
template int gemv_row_launch<double>(const GemvArgs<double>&, const GemvPlan&, cudaStream_t);

}  // namespace gb
