// Column-major GEMV, c_i <- c_i + alpha * sum_j A[i + j*lda] x_j.
//
// Alg. 1 of the paper (Sec. 4.1) blocks rows by m_c, columns by n_c and
// updates a short run of c, c(i_r : i_r + m_r), from a block of A and the
// matching block of x (its micro-kernel).  With 16-byte aligned operands a
// block tile is TX*V rows by a chunk of columns (gemv_col_tile_kernel, up to
// 256 row threads when the columns are few).  For misaligned operands
// (scalar loads) a warp item is TXW*V rows
// (each lane owns V consecutive rows, one 16-byte pack per column: the m_r
// of the micro-kernel) by a chunk of KC columns (n_c), walked by TYW =
// 32/TXW column lanes, so one load instruction of the warp reads TYW column
// segments of TXW*16 bytes.  The TYW partial vectors are summed by a fixed
// butterfly of shuffles; when the columns are split into S > 1 chunks the
// chunk partials are summed in a fixed order by the warp that finishes a row
// item last.  Warps work on items independently (grid-stride over items).
#include <mutex>

#include <cooperative_groups.h>

#include "gb_common.cuh"
#include "gb_internal.h"

namespace gb {
namespace {

// Sum over the lanes that share lane % TXW (offsets 16, 8, ..., TXW), in a
// fixed order; every lane ends with its group's total.
template <int TXW>
__device__ __forceinline__ double sum_over_ty(double v) {
#pragma unroll
  for (int o = 16; o >= TXW; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
template <int TXW>
__device__ __forceinline__ float sum_over_ty_f(float v) {
#pragma unroll
  for (int o = 16; o >= TXW; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

template <typename T, int V, int TXW, int U, bool LONG>
__global__ void __launch_bounds__(kThreads, 3)
    gemv_col_kernel(int64_t m, int64_t n, T alpha, const T* __restrict__ A, int64_t lda,
                    const T* __restrict__ x, T* __restrict__ c, const Split sp, int64_t KC,
                    int64_t items) {
  constexpr int TYW = 32 / TXW;
  constexpr int ROWS = TXW * V;  // rows per warp item
  // LONG (FP32 only): a lane's chain would exceed 64 products per row, so its
  // FP32 partial moves into FP64 every FLUSH bodies
  constexpr int FLUSH = LONG ? (64 / U > 0 ? 64 / U : 1) : 1 << 30;

  const int S = sp.S;
  const int lane = threadIdx.x & 31;
  const int tx = lane % TXW;
  const int ty = lane / TXW;
  const int64_t nwarps = (int64_t)gridDim.x * (kThreads / 32);

  for (int64_t it = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5; it < items; it += nwarps) {
    const int64_t ri = it / S;
    const int s = (int)(it - ri * S);
    const int64_t rbase = ri * ROWS;
    const int64_t i0 = rbase + (int64_t)tx * V;
    const int64_t k0 = (int64_t)s * KC;
    const int64_t k1 = (k0 + KC < n) ? k0 + KC : n;
    const bool full = i0 + V <= m;

    T acc[V];
    double tot[V];
#pragma unroll
    for (int v = 0; v < V; ++v) { acc[v] = T(0); tot[v] = 0.0; }

    const int64_t cstep = (int64_t)TYW * lda;  // pointer step between a lane's columns
    if (full) {
      const T* pa = A + i0 + (k0 + ty) * lda;   // this lane's pack of column k0 + ty
      const T* px = x + k0 + ty;
      int64_t j = k0 + ty;
      int body = 0;
#pragma unroll 1
      for (; j + (int64_t)(U - 1) * TYW < k1; j += (int64_t)U * TYW) {
        Pack<T, V> ap[U];
        T xs[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
          xs[q] = __ldg(px + q * TYW);
          ap[q] = ld_stream<T, V>(pa + q * cstep);
        }
        pa += U * cstep;
        px += U * TYW;
#pragma unroll
        for (int q = 0; q < U; ++q)
#pragma unroll
          for (int v = 0; v < V; ++v) acc[v] = fma_rn(ap[q].v[v], xs[q], acc[v]);
        if constexpr (LONG) {
          if (++body == FLUSH) {
            body = 0;
#pragma unroll
            for (int v = 0; v < V; ++v) { tot[v] = __dadd_rn(tot[v], (double)acc[v]); acc[v] = T(0); }
          }
        }
      }
#pragma unroll 1
      for (; j < k1; j += TYW, pa += cstep, px += TYW) {
        const T xs = __ldg(px);
        const Pack<T, V> ap = ld_stream<T, V>(pa);
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = fma_rn(ap.v[v], xs, acc[v]);
      }
    } else if (i0 < m) {  // the rows of the last item stop inside this lane's pack
      const T* pa = A + i0 + (k0 + ty) * lda;
      int body = 0;
      for (int64_t j = k0 + ty; j < k1; j += TYW, pa += cstep) {
        const T xs = __ldg(x + j);
#pragma unroll
        for (int v = 0; v < V; ++v)
          if (i0 + v < m) acc[v] = fma_rn(__ldcs(pa + v), xs, acc[v]);
        if constexpr (LONG) {
          if (++body == 64) {
            body = 0;
#pragma unroll
            for (int v = 0; v < V; ++v) { tot[v] = __dadd_rn(tot[v], (double)acc[v]); acc[v] = T(0); }
          }
        }
      }
    }

#pragma unroll
    for (int v = 0; v < V; ++v) {
      if constexpr (sizeof(T) == 4 && !LONG) tot[v] = (double)sum_over_ty_f<TXW>(acc[v]);
      else tot[v] = sum_over_ty<TXW>(__dadd_rn(tot[v], (double)acc[v]));
    }

    if (S == 1) {
      if (ty == 0) {
#pragma unroll
        for (int v = 0; v < V; ++v)
          if (i0 + v < m) c[i0 + v] = update_from(c[i0 + v], alpha, tot[v]);
      }
    } else {
      if (ty == 0) {
#pragma unroll
        for (int v = 0; v < V; ++v)
          if (i0 + v < m) sp.part[(int64_t)s * m + i0 + v] = tot[v];
      }
      const int rows = (int)((m - rbase < ROWS) ? m - rbase : ROWS);
      warp_split_finish<T>(sp, ri, s, rbase, rows, c, alpha);
    }
  }
}

// The last cluster's sum of the S cluster partials of rows [0, rows): CTA
// `rank` takes the rows rank*RPC .. rank*RPC + RPC - 1 (RPC = rows / CL,
// rounded up); thread t works on row t % P of them (P = RPC rounded up to
// a power of two, at most 32) and on slice t / P of the partials, which it
// sums in index order (loads issued together); the 32 / P slices of a row
// in a warp are added by a fixed xor butterfly, the 8 warps' sums in warp
// order, and c <- c0 + alpha * sum.  Every thread of the CTA calls it.
template <typename T, int CL>
__device__ __noinline__ void cluster_final_sum(const Split& sp, int rank, int rows, T* c, T alpha,
                                               const T* cpre, double* red) {
  const int rpc = (rows + CL - 1) / CL;
  const int r0 = rank * rpc;
  const int nr = r0 + rpc <= rows ? rpc : (rows > r0 ? rows - r0 : 0);
  if (nr <= 0) return;
  int p2 = 1;
  while (p2 < rpc) p2 <<= 1;
  const int ns = kThreads / p2;  // slices per row
  const int per = (sp.S + ns - 1) / ns;
  const int r = threadIdx.x % p2, j = threadIdx.x / p2;
  double acc = 0.0;
  if (r < nr) {
    const int q0 = j * per, q1 = q0 + per < sp.S ? q0 + per : sp.S;
    const double* p = sp.part + r0 + r;
    for (int qb = q0; qb < q1; qb += 8) {
      double v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = qb + k < q1 ? __ldcg(p + (int64_t)(qb + k) * sp.m) : 0.0;
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (qb + k < q1) acc = __dadd_rn(acc, v[k]);
    }
  }
  for (int o = 16; o >= p2; o >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
  const int lane = threadIdx.x & 31;
  if (lane < p2) red[(threadIdx.x >> 5) * p2 + lane] = acc;
  __syncthreads();
  if (threadIdx.x < nr) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) t = __dadd_rn(t, red[w * p2 + threadIdx.x]);
    c[r0 + threadIdx.x] = update_from(cpre[r0 + threadIdx.x], alpha, t);
  }
}

// 16-byte aligned operands: block tiles.  A work unit is a tile of RT = TX*V
// rows by a chunk of KC columns; thread (tx, ty) owns rows tx*V .. tx*V+V-1
// of the tile (one 16-byte pack per column) and every TY-th column of the
// chunk, with U packs in flight.  Block b takes the units b, b + G,
// b + 2G, ... (G blocks), so that at any moment the blocks read one compact
// window of memory that moves through A (measured on GB300: a higher
// stream rate and a shorter start than a contiguous range per block).  The TY partial vectors are summed
// through shared memory in ty order; S > 1 chunk partials are combined by
// block_split_finish.  FP32 sums stay in FP32 (chains of at most 64
// products, then a compensated FP32 sum).
//
// With CL > 0 (one row tile, the columns split into `units` chunks, a launch
// in thread-block clusters of CL CTAs) each CTA streams one chunk; the CTAs
// of a cluster leave their partial vectors in shared memory, CTA rank 0 sums
// them in rank order through distributed shared memory (the cluster barrier
// is hardware: every CTA of a cluster runs at once) and writes one partial
// per cluster, and the last cluster to finish sums those in cluster order.
template <typename T, int V, int TX, int U, bool LONG, int CL>
__global__ void __launch_bounds__(kThreads, 4)
    gemv_col_tile_kernel(int64_t m, int64_t n, T alpha, const T* __restrict__ A, int64_t lda,
                         const T* __restrict__ x, T* __restrict__ c, const Split sp, int64_t KC,
                         int64_t units) {
  constexpr int TY = kThreads / TX;
  constexpr int RT = TX * V;  // rows per tile
  constexpr int FLUSH = LONG ? (64 / U > 0 ? 64 / U : 1) : 1 << 30;
  // FP64: columns on the FP64 pipe per iteration (tiles of 128 or more rows
  // occur only with few columns, where more emulation measured faster)
  constexpr int DU = sizeof(T) == 8 ? (TX >= 128 ? kColTileD64Short : kColTileD64) : U;
  constexpr int NEM = U > DU ? U - DU : 1;  // emulated columns per iteration (1 when none)
  constexpr int EFLUSH = kEmuChain / NEM > 0 ? kEmuChain / NEM : 1;
  __shared__ T redT[kThreads * V];
  __shared__ double red_d[kThreads];
  __shared__ double cpart[CL > 0 ? TX * V : 1];  // CL: this CTA's partial vector
  __shared__ T cpre[CL > 0 ? TX * V : 1];         // CL: c of the tile's rows
  __shared__ int flag;

  const int tx = threadIdx.x % TX;
  const int ty = threadIdx.x / TX;
  const int S = CL > 0 ? (int)units : sp.S;  // column chunks per row tile
  const int64_t cstep = (int64_t)TY * lda;  // between a thread's columns

  // CL: c of the tile's rows (one per thread) copied into shared memory
  // while the columns stream, so that the final update waits on no load of c
  if constexpr (CL > 0) {
    static_assert(TX * V <= kThreads, "a cluster tile has at most one row per thread");
    if (threadIdx.x < RT && threadIdx.x < m) cp_async_elem(&cpre[threadIdx.x], c + threadIdx.x);
    cp_async_commit();
  }

  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {  // interleaved units
    const int64_t rt = u / S;
    const int s = (int)(u - rt * S);
    const int64_t i0 = rt * RT + (int64_t)tx * V;
    const int64_t k0 = (int64_t)s * KC;
    const int64_t k1 = (k0 + KC < n) ? k0 + KC : n;

    T acc[V], hi[V], lo[V];
    float eh[V], el[V];  // FP64: pairs of the FP32-emulated products
#pragma unroll
    for (int v = 0; v < V; ++v) { acc[v] = T(0); hi[v] = T(0); lo[v] = T(0); eh[v] = 0.f; el[v] = 0.f; }
    int ebody = 0;

    if (i0 + V <= m) {
      const T* pa = A + i0 + (k0 + ty) * lda;
      int64_t j = k0 + ty;
      int body = 0;
#pragma unroll 1
      for (; j + (int64_t)(U - 1) * TY < k1; j += (int64_t)U * TY) {
        Pack<T, V> ap[U];
        T xs[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
          ap[q] = ld_stream<T, V>(pa + q * cstep);
          xs[q] = __ldg(x + j + q * TY);
        }
        pa += U * cstep;
        if constexpr (sizeof(T) == 8) {
          // FP64: the first DU columns on the FP64 pipe, the others with
          // FP32 instructions (emu_fma) into the pairs (eh, el)
#pragma unroll
          for (int q = 0; q < DU; ++q)
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] = fma_rn(ap[q].v[v], xs[q], acc[v]);
          unsigned rb = 0u;  // the emulated operands' ranges, OR-ed
#pragma unroll
          for (int q = DU; q < U; ++q) {
            rb |= emu_range(xs[q]);
#pragma unroll
            for (int v = 0; v < V; ++v) rb |= emu_range(ap[q].v[v]);
          }
          const bool ok = rb < kEmuRange;
          // the choice is made for all the lanes that run here together (the
          // active mask: lanes of one warp may leave this loop at different
          // trips), so that the emulated path holds no FP64 instruction (a
          // predicated-off one would still occupy the FP64 pipe)
          if (__all_sync(__activemask(), ok)) {
#pragma unroll
            for (int q = DU; q < U; ++q) {
              float xh, xl;
              emu_split(xs[q], xh, xl);
#pragma unroll
              for (int v = 0; v < V; ++v) {
                float ah, al;
                emu_split(ap[q].v[v], ah, al);
                emu_fma(ah, al, xh, xl, eh[v], el[v]);
              }
            }
          } else {
#pragma unroll
            for (int v = 0; v < V; ++v) {
              DPacks<U - DU> dp;
#pragma unroll
              for (int q = DU; q < U; ++q) {
                dp.a[q - DU] = ap[q].v[v];
                dp.x[q - DU] = xs[q];
              }
              acc[v] = dfma_fallback(dp, acc[v]);
            }
          }
          if (++ebody == EFLUSH) {  // at most kEmuChain products per row in the FP32 pairs
            ebody = 0;
#pragma unroll
            for (int v = 0; v < V; ++v) emu_fold(acc[v], eh[v], el[v]);
          }
        } else {
#pragma unroll
          for (int q = 0; q < U; ++q)
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] = fma_rn(ap[q].v[v], xs[q], acc[v]);
        }
        if constexpr (LONG) {
          if (++body == FLUSH) {
            body = 0;
#pragma unroll
            for (int v = 0; v < V; ++v) {
              float e;
              two_sum_f(hi[v], acc[v], hi[v], e);
              lo[v] = __fadd_rn(lo[v], e);
              acc[v] = T(0);
            }
          }
        }
      }
#pragma unroll 1
      for (; j < k1; j += TY, pa += cstep) {
        const Pack<T, V> ap = ld_stream<T, V>(pa);
        const T xs = __ldg(x + j);
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = fma_rn(ap.v[v], xs, acc[v]);
      }
    } else if (i0 < m) {  // the last rows of the matrix stop inside this thread's pack
      int body = 0;
      for (int64_t j = k0 + ty; j < k1; j += TY) {
        const T xs = __ldg(x + j);
#pragma unroll
        for (int v = 0; v < V; ++v)
          if (i0 + v < m) acc[v] = fma_rn(__ldcs(A + i0 + v + j * lda), xs, acc[v]);
        if constexpr (LONG) {
          if (++body == 64) {
            body = 0;
#pragma unroll
            for (int v = 0; v < V; ++v) {
              float e;
              two_sum_f(hi[v], acc[v], hi[v], e);
              lo[v] = __fadd_rn(lo[v], e);
              acc[v] = T(0);
            }
          }
        }
      }
    }
    if constexpr (LONG) {
#pragma unroll
      for (int v = 0; v < V; ++v) acc[v] = hi[v] + (lo[v] + acc[v]);
    }
    if constexpr (sizeof(T) == 8) {
#pragma unroll
      for (int v = 0; v < V; ++v) emu_fold(acc[v], eh[v], el[v]);
    }

    // CL (TX < 32): the 32 / TX column lanes of a warp are first added by a
    // fixed xor butterfly, so that the shared-memory sum has one entry per
    // warp and row instead of one per column lane
    constexpr bool WB = CL > 0 && TX < 32;
    constexpr int NY = WB ? kThreads / 32 : TY;  // entries per row in redT
    __syncthreads();  // redT is free
    if constexpr (WB) {
#pragma unroll
      for (int v = 0; v < V; ++v)
#pragma unroll
        for (int o = 16; o >= TX; o >>= 1) acc[v] = acc[v] + __shfl_xor_sync(0xffffffffu, acc[v], o);
      if ((threadIdx.x & 31) < TX)
#pragma unroll
        for (int v = 0; v < V; ++v) redT[(threadIdx.x >> 5) * RT + tx * V + v] = acc[v];
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) redT[ty * RT + tx * V + v] = acc[v];
    }
    __syncthreads();
    for (int r = threadIdx.x; r < RT; r += kThreads) {
      T t = T(0);
      for (int y = 0; y < NY; ++y) t = t + redT[y * RT + r];
      const int64_t row = rt * RT + r;
      if constexpr (CL > 0) {
        cpart[r] = (double)t;
      } else if (row < m) {
        if (S == 1) c[row] = update(c[row], alpha, t);
        else sp.part[(int64_t)s * m + row] = (double)t;
      }
    }
    if constexpr (CL > 0) {
      namespace cg = cooperative_groups;
      cg::cluster_group cluster = cg::this_cluster();
      cp_async_wait<0>();  // this thread's row of cpre (read only by this thread or after a barrier)
      cluster.sync();  // every CTA of the cluster holds its partial vector
      const bool lead = cluster.block_rank() == 0;
      const int64_t q = blockIdx.x / CL;  // the cluster's partial
      if (lead) {
        for (int r = threadIdx.x; r < RT && r < m; r += kThreads) {
          double v = 0.0;
#pragma unroll
          for (int k = 0; k < CL; ++k) v = __dadd_rn(v, *cluster.map_shared_rank(&cpart[r], k));
          if (sp.S == 1) c[r] = update_from(cpre[r], alpha, v);
          else sp.part[q * m + r] = v;
        }
        if (sp.S > 1) {
          // the cluster's arrival, told to every CTA of the cluster
          __syncthreads();  // the cluster partial is written (released by the increment)
          if (threadIdx.x == 0) {
            const int last = arrive_add(sp.tickets) == (unsigned)sp.S - 1;
#pragma unroll
            for (int k = 0; k < CL; ++k) *cluster.map_shared_rank(&flag, k) = last;
            if (last) *sp.tickets = 0u;  // every cluster has arrived
          }
        }
      }
      // rank 0 has read every partial vector and written every flag; no CTA
      // leaves before that
      cluster.sync();
      if (sp.S > 1 && flag) {
        // the last cluster: CTA k sums the cluster partials of its share of
        // the rows, all of its loads in one round trip
        fence_acq_rel_gpu();  // (the cluster barrier carries rank 0's acquire; made explicit)
        cluster_final_sum<T, CL>(sp, (int)cluster.block_rank(), m < RT ? (int)m : RT, c, alpha, cpre, red_d);
      }
    } else if (S > 1) {
      const int64_t t0 = rt * RT;
      block_split_finish<T>(sp, rt, s, t0, (m - t0 < RT) ? m - t0 : RT, c, alpha, red_d, &flag);
    }
  }
}

// Clusters of kColCluster CTAs of `kern` resident at once on the current
// device (queried once per kernel and device).
int cluster_capacity(const void* kern) {
  struct Entry {
    const void* k;
    int dev, clusters;
  };
  static Entry cache[64];
  static int used = 0;
  static std::mutex mu;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  for (int i = 0; i < used; ++i)
    if (cache[i].k == kern && cache[i].dev == dev) return cache[i].clusters;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kColCluster * 1024);
  cfg.blockDim = dim3(kThreads);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kColCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess || n < 1) n = 1;
  if (used < 64) cache[used++] = Entry{kern, dev, n};
  return n;
}

// One CTA per column chunk in clusters of kColCluster.  The plan's chunk
// count is capped here at the clusters the device runs at once (a second
// wave would double the time): fewer, longer chunks, and as many cluster
// partials as clusters (the workspace, sized for the plan's count, holds
// them); FP32 chains past 64 products per thread take the LONG form.  The
// last cluster to arrive sums the cluster partials with all of its CTAs.
template <typename T, int V, int TX>
int launch_cluster(const GemvArgs<T>& a, const GemvPlan& p, cudaStream_t st) {
  constexpr int TY = kThreads / TX;
  constexpr int U = sizeof(T) == 4 ? kColClusterU32 : kColTileU;
  auto k0 = gemv_col_tile_kernel<T, V, TX, U, false, kColCluster>;
  auto k1 = gemv_col_tile_kernel<T, V, TX, U, sizeof(T) == 4, kColCluster>;
  int64_t parts = p.units / kColCluster;
  const int cap = cluster_capacity((const void*)k0);
  if (parts > cap) parts = cap;
  const int64_t chunks = parts * kColCluster;
  const int64_t kc = (a.n + chunks - 1) / chunks;
  Split sp = p.split;
  sp.S = sp.G = (int)parts;
  sp.NG = 1;
  const bool longc = sizeof(T) == 4 && (kc + TY - 1) / TY > 64;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)chunks);
  cfg.blockDim = dim3(kThreads);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kColCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (longc)
    cudaLaunchKernelEx(&cfg, k1, a.m, a.n, a.alpha, a.A, a.lda, a.x, a.c, sp, kc, chunks);
  else
    cudaLaunchKernelEx(&cfg, k0, a.m, a.n, a.alpha, a.A, a.lda, a.x, a.c, sp, kc, chunks);
  return 0;
}

template <typename T, int V, int TX, bool LONG>
int launch_tile(const GemvArgs<T>& a, const GemvPlan& p, cudaStream_t st) {
  if constexpr (TX * V <= 256) {
    if (p.cluster == kColCluster) return launch_cluster<T, V, TX>(a, p, st);
  }
  auto kern = gemv_col_tile_kernel<T, V, TX, kColTileU, LONG, 0>;
  const int grid = grid_size((const void*)kern, p.units, 0, sizeof(T) == 8 ? kColTileWaves64 : 1);
  kern<<<grid, kThreads, 0, st>>>(a.m, a.n, a.alpha, a.A, a.lda, a.x, a.c, p.split, p.kc, p.units);
  return 0;
}

template <typename T, int V, int TXW, bool LONG>
int launch(const GemvArgs<T>& a, const GemvPlan& p, cudaStream_t st) {
  auto kern = gemv_col_kernel<T, V, TXW, 8, LONG>;
  const int64_t blocks = (p.units + kThreads / 32 - 1) / (kThreads / 32);
  const int grid = grid_size((const void*)kern, blocks);
  kern<<<grid, kThreads, 0, st>>>(a.m, a.n, a.alpha, a.A, a.lda, a.x, a.c, p.split, p.kc, p.units);
  return 0;
}

template <typename T, int V, bool LONG>
int by_txw(const GemvArgs<T>& a, const GemvPlan& p, cudaStream_t st) {
  if constexpr (V > 1) {  // 16-byte aligned operands: block tiles (tx = threads along the rows)
    switch (p.txw) {
      case 256: return launch_tile<T, V, 256, LONG>(a, p, st);
      case 128: return launch_tile<T, V, 128, LONG>(a, p, st);
      case 64: return launch_tile<T, V, 64, LONG>(a, p, st);
      case 32: return launch_tile<T, V, 32, LONG>(a, p, st);
      case 16: return launch_tile<T, V, 16, LONG>(a, p, st);
      case 8: return launch_tile<T, V, 8, LONG>(a, p, st);
      case 4: return launch_tile<T, V, 4, LONG>(a, p, st);
      case 2: return launch_tile<T, V, 2, LONG>(a, p, st);
      default: return launch_tile<T, V, 1, LONG>(a, p, st);
    }
  } else {
    switch (p.txw) {
      case 32: return launch<T, V, 32, LONG>(a, p, st);
      case 16: return launch<T, V, 16, LONG>(a, p, st);
      case 8: return launch<T, V, 8, LONG>(a, p, st);
      case 4: return launch<T, V, 4, LONG>(a, p, st);
      case 2: return launch<T, V, 2, LONG>(a, p, st);
      default: return launch<T, V, 1, LONG>(a, p, st);
    }
  }
}

}  // namespace

template <typename T>
int gemv_col_launch(const GemvArgs<T>& a, const GemvPlan& p, cudaStream_t st) {
  constexpr int V = 16 / sizeof(T);
  if constexpr (sizeof(T) == 4) {
    if (p.vec) return p.long_chain ? by_txw<T, V, true>(a, p, st) : by_txw<T, V, false>(a, p, st);
    return p.long_chain ? by_txw<T, 1, true>(a, p, st) : by_txw<T, 1, false>(a, p, st);
  } else {
    if (p.vec) return by_txw<T, V, false>(a, p, st);
    return by_txw<T, 1, false>(a, p, st);
  }
}

template int gemv_col_launch<float>(const GemvArgs<float>&, const GemvPlan&, cudaStream_t);
template int gemv_col_launch<double>(const GemvArgs<double>&, const GemvPlan&, cudaStream_t);

}  // namespace gb
