// Column-major GEMV, c_i <- c_i + alpha * sum_j A[i + j*lda] x_j.
//
// Alg. 1 of the paper (Sec. 4.1) blocks rows by m_c, columns by n_c and
// updates a short run of c, c(i_r : i_r + m_r), from a block of A and the
// matching block of x (its micro-kernel).  Here a block tile is TX*V rows
// (each thread owns V consecutive rows, moved as one 16-byte pack per
// column: the m_r of the micro-kernel) by a chunk of KC columns (n_c),
// walked by TY = 256/TX column lanes.  The TY partial vectors are summed in
// shared memory in lane order; when the columns are split into S > 1
// chunks the chunk partials are summed in a fixed order by the block that
// finishes a row tile last.
#include "gb_common.cuh"
#include "gb_internal.h"

namespace gb {
namespace {

template <typename T, int V, int TX, int U>
__global__ void __launch_bounds__(kThreads)
    gemv_col_kernel(int64_t m, int64_t n, T alpha, const T* __restrict__ A, int64_t lda,
                    const T* __restrict__ x, T* __restrict__ c, const Split sp, int64_t KC,
                    int64_t units) {
  const int S = sp.S;
  constexpr int TY = kThreads / TX;
  constexpr int RT = TX * V;  // rows per tile
  constexpr int FLUSH = (sizeof(T) == 4) ? (64 / U > 0 ? 64 / U : 1) : 1 << 30;

  __shared__ double red[kThreads * V];
  __shared__ int flag;

  const int tx = threadIdx.x % TX;
  const int ty = threadIdx.x / TX;

  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int64_t rt = u / S;
    const int s = (int)(u - rt * S);
    const int64_t i0 = rt * RT + (int64_t)tx * V;
    const int64_t k0 = (int64_t)s * KC;
    const int64_t k1 = (k0 + KC < n) ? k0 + KC : n;
    const bool full = i0 + V <= m;
    const bool any = i0 < m;
    const T* Ai = A + (any ? i0 : 0);

    T acc[V];
    double tot[V];
#pragma unroll
    for (int v = 0; v < V; ++v) { acc[v] = T(0); tot[v] = 0.0; }

    auto load = [&](int64_t j) {
      Pack<T, V> p;
      if (full) {
        p = ld_stream<T, V>(Ai + j * lda);
      } else {
#pragma unroll
        for (int v = 0; v < V; ++v) p.v[v] = (i0 + v < m) ? __ldcs(Ai + v + j * lda) : T(0);
      }
      return p;
    };

    int64_t j = k0 + ty;
    int body = 0;
    if (any) {
      for (; j + (int64_t)(U - 1) * TY < k1; j += (int64_t)U * TY) {
        Pack<T, V> ap[U];
        T xs[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
          xs[q] = __ldg(x + j + q * TY);
          ap[q] = load(j + q * TY);
        }
#pragma unroll
        for (int q = 0; q < U; ++q)
#pragma unroll
          for (int v = 0; v < V; ++v) acc[v] = fma_rn(ap[q].v[v], xs[q], acc[v]);
        if constexpr (sizeof(T) == 4) {
          if (++body == FLUSH) {
            body = 0;
#pragma unroll
            for (int v = 0; v < V; ++v) { tot[v] = __dadd_rn(tot[v], (double)acc[v]); acc[v] = 0.f; }
          }
        }
      }
      for (; j < k1; j += TY) {
        const T xs = __ldg(x + j);
        const Pack<T, V> ap = load(j);
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = fma_rn(ap.v[v], xs, acc[v]);
      }
    }
#pragma unroll
    for (int v = 0; v < V; ++v) red[ty * RT + tx * V + v] = __dadd_rn(tot[v], (double)acc[v]);
    __syncthreads();
    for (int r = threadIdx.x; r < RT; r += kThreads) {
      const int64_t row = rt * RT + r;
      double t = 0.0;
      for (int y = 0; y < TY; ++y) t = __dadd_rn(t, red[y * RT + r]);
      if (row < m) {
        if (S == 1) c[row] = update(c[row], alpha, t);
        else sp.part[(int64_t)s * m + row] = t;
      }
    }
    __syncthreads();
    if (S > 1) {
      const int64_t t0 = rt * RT;
      split_finish<T>(sp, rt, s, t0, (m - t0 < RT) ? m - t0 : RT, c, alpha, red, &flag);
    }
  }
}

template <typename T, int V, int TX>
int launch(const GemvArgs<T>& a, const GemvPlan& p, cudaStream_t st) {
  auto kern = gemv_col_kernel<T, V, TX, 4>;
  const int grid = grid_size((const void*)kern, p.units);
  kern<<<grid, kThreads, 0, st>>>(a.m, a.n, a.alpha, a.A, a.lda, a.x, a.c, p.split, p.kc, p.units);
  return 0;
}

template <typename T, int V>
int by_tx(const GemvArgs<T>& a, const GemvPlan& p, cudaStream_t st) {
  switch (p.tx) {
    case 64: return launch<T, V, 64>(a, p, st);
    case 32: return launch<T, V, 32>(a, p, st);
    case 16: return launch<T, V, 16>(a, p, st);
    case 8: return launch<T, V, 8>(a, p, st);
    case 4: return launch<T, V, 4>(a, p, st);
    case 2: return launch<T, V, 2>(a, p, st);
    default: return launch<T, V, 1>(a, p, st);
  }
}

}  // namespace

template <typename T>
int gemv_col_launch(const GemvArgs<T>& a, const GemvPlan& p, cudaStream_t st) {
  if (p.vec) return by_tx<T, 16 / sizeof(T)>(a, p, st);
  return by_tx<T, 1>(a, p, st);
}

template int gemv_col_launch<float>(const GemvArgs<float>&, const GemvPlan&, cudaStream_t);
template int gemv_col_launch<double>(const GemvArgs<double>&, const GemvPlan&, cudaStream_t);

}  // namespace gb
