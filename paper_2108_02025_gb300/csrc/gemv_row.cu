// Row-major GEMV, c_i <- c_i + alpha * sum_j A[i*lda + j] x_j.
//
// Alg. 2 of the paper (Sec. 4.2) hands each row, a unit-stride dot product,
// to one worker; Loop-1 (rows) is the parallel loop.  On the GPU the rows
// are streamed so that every block reads one contiguous stretch of memory:
//
// * long rows (more than 256 16-byte packs): a work unit is one chunk of KC
//   columns of one row (KC = n unless the rows are too few to fill the GPU,
//   when the columns are split into S chunks, the blocking of the index
//   range of Alg. 4).  Block b takes the units b, b + G, b + 2G, ... (G
//   blocks: the blocks read one compact window that moves through A, which
//   streams faster on GB300 than a contiguous range per block) and streams
//   each with all 256 threads
//   (16-byte loads, U packs per thread in flight), then sums the unit in a
//   fixed order (warp butterfly, then warps in order).  A split row's chunk
//   partials are summed in chunk order by the block that finishes the row.
// * short rows (at most 256 packs): LPR lanes share a row, each holding up to
//   8 of its packs, so a block iteration reads 256/LPR consecutive rows; the
//   LPR lanes of a row are summed by a butterfly.
// * FP64 long rows go in groups of two rows per unit (each load and FP32
//   cut of x serves both); part of every FP64 row's products are formed
//   with FP32 instructions (gb_common.cuh), since the FP64 pipe alone cannot
//   keep up with HBM on GB300.
// * FP32 rows are summed in FP32 throughout (chains of at most 64 products,
//   then a compensated FP32 sum); split partials are combined in FP64.
// * rows that do not start on 16 bytes (odd lda, or A offset by whole
//   elements) with x aligned: the same units, read in aligned packs and
//   realigned to x (shift kernels below).
// * x misaligned too (no 16-byte packs at all): warp items of RW rows with
//   scalar loads.
#include "gb_common.cuh"
#include "gb_internal.h"

namespace gb {
namespace {

// Sum of one value per thread over the block in a fixed order (warp
// butterfly, then the 8 warp totals in order), in the element type;
// the result is valid in thread 0.  Synchronises the block.
template <typename T>
__device__ __forceinline__ T block_total(T v, T* red) {
  if constexpr (sizeof(T) == 4) v = group_sum_f<32>(v);
  else v = group_sum<32>(v);
  __syncthreads();  // red is free (its previous use has been read)
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  T t = T(0);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < kThreads / 32; ++k) t = t + red[k];
  }
  return t;
}

// The final step of a split row, in the block that arrived last: the S
// chunk partials in FP64 (thread t adds chunks t, t+256, ... in order, then
// the fixed block order), c_row <- c0 + alpha * sum (c0, the row's c, is
// read in thread 0 only), and the row's counter back to zero.  Every thread
// of the block calls it.
template <typename T>
__device__ __forceinline__ void row_split_sum(const Split& sp, int64_t row, int S, T alpha, T* c, double c0,
                                              double* red_d) {
  double p = 0.0;
  for (int q = threadIdx.x; q < S; q += kThreads) p = __dadd_rn(p, __ldcg(sp.part + (int64_t)q * sp.m + row));
  const double sum = block_total<double>(p, red_d);
  if (threadIdx.x == 0) {
    c[row] = update_from((T)c0, alpha, sum);  // c0 holds a T exactly
    sp.tickets[row] = 0u;
  }
}

// Long rows.  unit u = (row u / S, chunk u % S).
template <typename T, int V, int U, bool LONG>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 8 ? kRowLongB64 : 4)
    gemv_row_long_kernel(int64_t m, int64_t n, T alpha, const T* __restrict__ A, int64_t lda,
                         const T* __restrict__ x, T* __restrict__ c, const Split sp, int64_t KC,
                         int64_t units) {
  constexpr int64_t STEP = (int64_t)kThreads * V;  // columns the block covers per pack
  // LONG (FP32 only): a thread's chain would exceed 64 products, so every
  // FLUSH bodies it is folded into a compensated FP32 sum (TwoSum)
  constexpr int FLUSH = LONG ? (64 / (U * V) > 0 ? 64 / (U * V) : 1) : 1 << 30;
  constexpr int UD = sizeof(T) == 8 ? (kRowLongD64 < U ? kRowLongD64 : U) : U;  // packs on the FP64 pipe
  constexpr int NEM = (U - UD) * V > 0 ? (U - UD) * V : 1;  // emulated products per iteration (1 when none)
  constexpr int EFLUSH = kEmuChain / NEM > 0 ? kEmuChain / NEM : 1;
  __shared__ double red_d[kThreads / 32];
  __shared__ int flag;
  // split rows: the block's first kRowHeld units have their arrival deferred
  // to the end of the block's work (row, prefetched c, and whether this
  // block finishes the row), so that no block stops streaming mid-kernel to
  // finish a row
  __shared__ int64_t hrow[kRowHeld];
  __shared__ double hc[kRowHeld];
  __shared__ int hlast[kRowHeld];
  T* red = reinterpret_cast<T*>(red_d);

  const int S = sp.S;
  int nheld = 0;
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {  // interleaved units
    const int64_t row = u / S;
    const int s = (int)(u - row * S);
    const int64_t k0 = (int64_t)s * KC;
    const int64_t k1 = (k0 + KC < n) ? k0 + KC : n;
    const int64_t kv1 = k0 + ((k1 - k0) / V) * V;
    const T* Ar = A + row * lda;
    // split rows: c of the row, read now so that a final update waits on no load
    T c0 = T(0);
    if (S > 1 && threadIdx.x == 0) c0 = c[row];

    T acc = T(0), acc2 = T(0), hi = T(0), lo = T(0);
    float eh = 0.f, el = 0.f;  // FP64: the pair of the FP32-emulated products
    int body = 0;
    int64_t j = k0 + (int64_t)threadIdx.x * V;
    // the main loop runs while the warp's last lane has U whole packs left,
    // so that all 32 lanes take the same number of trips
    const int64_t jlast = (int64_t)(31 - (threadIdx.x & 31)) * V;
#pragma unroll 1
    for (; j + jlast + (U - 1) * STEP < kv1; j += U * STEP) {
      Pack<T, V> ap[U], xp[U];
#pragma unroll
      for (int q = 0; q < U; ++q) ap[q] = ld_stream<T, V>(Ar + j + q * STEP);
#pragma unroll
      for (int q = 0; q < U; ++q) xp[q] = ld_keep<T, V>(x + j + q * STEP);
      if constexpr (sizeof(T) == 8) {
        // FP64: the first half of the packs on the FP64 pipe, the second
        // half with FP32 instructions (emu_fma) into the pair (eh, el).  The
        // choice is made for all the lanes running here together (the active
        // mask), so that the emulated path holds no FP64 instruction (a
        // predicated-off one would still occupy the FP64 pipe).
#pragma unroll
        for (int q = 0; q < UD; ++q)
#pragma unroll
          for (int v = 0; v < V; ++v) {  // two FP64 chains (v), half the dependent latency
            if (v == 0) acc = fma_rn(ap[q].v[v], xp[q].v[v], acc);
            else acc2 = fma_rn(ap[q].v[v], xp[q].v[v], acc2);
          }
        unsigned rb = 0u;  // the emulated operands' ranges, OR-ed
#pragma unroll
        for (int q = UD; q < U; ++q)
#pragma unroll
          for (int v = 0; v < V; ++v) rb |= emu_range(ap[q].v[v]) | emu_range(xp[q].v[v]);
        if (__all_sync(__activemask(), rb < kEmuRange)) {
#pragma unroll
          for (int q = UD; q < U; ++q)
#pragma unroll
            for (int v = 0; v < V; ++v) {
              float ah, al, xh, xl;
              emu_split(ap[q].v[v], ah, al);
              emu_split(xp[q].v[v], xh, xl);
              emu_fma(ah, al, xh, xl, eh, el);
            }
        } else {
          DPacks<(U - UD) * V> dp;
#pragma unroll
          for (int q = UD; q < U; ++q)
#pragma unroll
            for (int v = 0; v < V; ++v) {
              dp.a[(q - UD) * V + v] = ap[q].v[v];
              dp.x[(q - UD) * V + v] = xp[q].v[v];
            }
          acc = dfma_fallback(dp, acc);
        }
        if (++body == EFLUSH) {  // at most kEmuChain products in the FP32 pair
          body = 0;
          emu_fold(acc, eh, el);
        }
      } else {
#pragma unroll
        for (int q = 0; q < U; ++q)
#pragma unroll
          for (int v = 0; v < V; ++v) acc = fma_rn(ap[q].v[v], xp[q].v[v], acc);
        if constexpr (LONG) {
          if (++body == FLUSH) {
            body = 0;
            float e;
            two_sum_f(hi, acc, hi, e);
            lo = __fadd_rn(lo, e);
            acc = T(0);
          }
        }
      }
    }
#pragma unroll 1
    for (; j < kv1; j += STEP) {
      const Pack<T, V> ap = ld_stream<T, V>(Ar + j), xp = ld_keep<T, V>(x + j);
#pragma unroll
      for (int v = 0; v < V; ++v) acc = fma_rn(ap.v[v], xp.v[v], acc);
    }
    if (kv1 + threadIdx.x < k1) {  // ragged end (< V columns)
      const int64_t jj = kv1 + threadIdx.x;
      acc = fma_rn(__ldcs(Ar + jj), __ldg(x + jj), acc);
    }
    if constexpr (LONG) acc = hi + (lo + acc);
    if constexpr (sizeof(T) == 8) {
      acc = __dadd_rn(acc, acc2);
      emu_fold(acc, eh, el);
    }

    const T total = block_total<T>(acc, red);
    if (S == 1) {
      if (threadIdx.x == 0) c[row] = update(c[row], alpha, total);
    } else {
      if (threadIdx.x == 0) sp.part[(int64_t)s * m + row] = (double)total;
      if (nheld < kRowHeld) {  // arrival deferred (block-uniform count)
        if (threadIdx.x == 0) {
          hrow[nheld] = row;
          hc[nheld] = (double)c0;
        }
        ++nheld;
      } else if (arrive_last(sp.tickets + row, (unsigned)S, &flag)) {
        row_split_sum(sp, row, S, alpha, c, (double)c0, red_d);  // (c0 is read in thread 0 only)
      }
    }
  }
  if (nheld > 0) {  // the deferred arrivals, all at once: thread k arrives for entry k
    __syncthreads();  // the partials and the entries are written
    if (threadIdx.x < nheld) hlast[threadIdx.x] = arrive_add(sp.tickets + hrow[threadIdx.x]) == (unsigned)S - 1;
    __syncthreads();  // the last arrival's partial reads come after its increment
    for (int k = 0; k < nheld; ++k)
      if (hlast[k]) row_split_sum(sp, hrow[k], S, alpha, c, hc[k], red_d);
  }
}

// The last block to finish a chunk of row group `grp` (rows row0 ..
// row0 + R - 1) sums each row's S chunk partials: thread t adds chunks t,
// t+256, ... in order, then the fixed block order; out of line, so that the
// streaming loop keeps its registers.  Every thread of the block calls it.
__device__ __noinline__ void multi_split_finish(const Split sp, int64_t grp, int64_t row0, int R, int64_t m,
                                                double alpha, double* __restrict__ c, double* red, int* flag) {
  const int S = sp.S;
  if (!arrive_last(sp.tickets + grp, (unsigned)S, flag)) return;
  for (int r = 0; r < R && row0 + r < m; ++r) {
    double p = 0.0;
    for (int q = threadIdx.x; q < S; q += kThreads) p = __dadd_rn(p, __ldcg(sp.part + (int64_t)q * m + row0 + r));
    p = group_sum<32>(p);
    __syncthreads();  // red is free
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = p;
    __syncthreads();
    if (threadIdx.x == 0) {
      double sum = 0.0;
#pragma unroll
      for (int w = 0; w < kThreads / 32; ++w) sum = sum + red[w];
      c[row0 + r] = update_from(c[row0 + r], alpha, sum);
    }
  }
  if (threadIdx.x == 0) sp.tickets[grp] = 0u;
}

// Row-major long rows that do not start on a 16-byte boundary (lda not a
// multiple of the pack, or A itself offset by whole elements), x 16-byte
// aligned.  A row is read in 16-byte packs from the aligned address below
// it: the columns [tV, tV+V) are the last V - MIS elements of aligned pack t
// and the first MIS of pack t+1 (both inside the row; MIS is the row's
// offset in elements, the same for every lane), so A and x line up again;
// the first column pack and the row's end are read element by element.
// Units, blocks, chains and sums as in the long-row kernel; FP64 products
// all on the FP64 pipe.
template <typename T, int V, int MIS, int U, bool LONG>
__device__ __forceinline__ T shift_packs(const T* __restrict__ Ab, const T* __restrict__ x, int64_t tv0,
                                         int64_t tv1) {
  constexpr int64_t SP = kThreads;  // packs per block pass
  constexpr int FLUSH = LONG ? (64 / (U * V) > 0 ? 64 / (U * V) : 1) : 1 << 30;
  T acc = T(0), hi = T(0), lo = T(0);
  int body = 0;
  int64_t t = tv0 + threadIdx.x;
#pragma unroll 1
  for (; t + (U - 1) * SP < tv1; t += U * SP) {
    Pack<T, V> a0[U], a1[U], xp[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      a0[q] = ld_stream<T, V>(Ab + (t + q * SP) * V);
      if constexpr (MIS > 0) a1[q] = ld_keep<T, V>(Ab + (t + q * SP + 1) * V);  // the neighbour lane's pack
      xp[q] = ld_keep<T, V>(x + (t + q * SP) * V);
    }
#pragma unroll
    for (int q = 0; q < U; ++q)
#pragma unroll
      for (int v = 0; v < V; ++v) {
        T a;
        if constexpr (MIS > 0) a = v + MIS < V ? a0[q].v[v + MIS] : a1[q].v[v + MIS - V];
        else a = a0[q].v[v];
        acc = fma_rn(a, xp[q].v[v], acc);
      }
    if constexpr (LONG) {
      if (++body == FLUSH) {
        body = 0;
        float e;
        two_sum_f(hi, acc, hi, e);
        lo = __fadd_rn(lo, e);
        acc = T(0);
      }
    }
  }
#pragma unroll 1
  for (; t < tv1; t += SP) {
    const Pack<T, V> a0 = ld_stream<T, V>(Ab + t * V);
    Pack<T, V> a1;
    if constexpr (MIS > 0) a1 = ld_keep<T, V>(Ab + (t + 1) * V);
    const Pack<T, V> xp = ld_keep<T, V>(x + t * V);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      T a;
      if constexpr (MIS > 0) a = v + MIS < V ? a0.v[v + MIS] : a1.v[v + MIS - V];
      else a = a0.v[v];
      acc = fma_rn(a, xp.v[v], acc);
    }
  }
  if constexpr (LONG) acc = hi + (lo + acc);
  return acc;
}

template <typename T, int V, int U, bool LONG>
__global__ void __launch_bounds__(kThreads, 4)
    gemv_row_shift_kernel(int64_t m, int64_t n, T alpha, const T* __restrict__ A, int64_t lda,
                          const T* __restrict__ x, T* __restrict__ c, const Split sp, int64_t KC,
                          int64_t units) {
  __shared__ double red_d[kThreads / 32];
  __shared__ int flag;
  T* red = reinterpret_cast<T*>(red_d);
  const int S = sp.S;
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {  // interleaved units
    const int64_t row = u / S;
    const int s = (int)(u - row * S);
    const int64_t k0 = (int64_t)s * KC;  // a multiple of V
    const int64_t k1 = (k0 + KC < n) ? k0 + KC : n;
    const T* Ar = A + row * lda;
    const int mis = (int)((reinterpret_cast<uintptr_t>(Ar) / sizeof(T)) % V);
    const T* Ab = Ar - mis;  // 16-byte aligned
    // column packs read as vectors: inside [k0, k1), and (MIS > 0) pack t+1
    // of the aligned base still inside the row, pack t not before it
    int64_t tv0 = k0 / V, tv1 = k1 / V;
    if (mis > 0) {
      if (tv0 < 1) tv0 = 1;
      const int64_t lim = (mis + n) / V - 1;
      if (tv1 > lim) tv1 = lim;
    }
    if (tv1 < tv0) tv1 = tv0;
    T acc;
    switch (mis) {
      case 0: acc = shift_packs<T, V, 0, U, LONG>(Ab, x, tv0, tv1); break;
      case 1: acc = shift_packs<T, V, 1, U, LONG>(Ab, x, tv0, tv1); break;
      case 2: acc = shift_packs<T, V, (V > 2 ? 2 : 1), U, LONG>(Ab, x, tv0, tv1); break;
      default: acc = shift_packs<T, V, (V > 3 ? 3 : 1), U, LONG>(Ab, x, tv0, tv1); break;
    }
    // the columns outside the vector packs, element by element
    for (int64_t col = k0 + threadIdx.x; col < tv0 * V && col < k1; col += kThreads)
      acc = fma_rn(__ldcs(Ar + col), __ldg(x + col), acc);
    for (int64_t col = (tv1 * V > k0 ? tv1 * V : k0) + threadIdx.x; col < k1; col += kThreads)
      if (col >= tv0 * V) acc = fma_rn(__ldcs(Ar + col), __ldg(x + col), acc);

    const T total = block_total<T>(acc, red);
    if (S == 1) {
      if (threadIdx.x == 0) c[row] = update(c[row], alpha, total);
    } else {
      if (threadIdx.x == 0) sp.part[(int64_t)s * m + row] = (double)total;
      if (arrive_last(sp.tickets + row, (unsigned)S, &flag)) {
        double p = 0.0;
        for (int q = threadIdx.x; q < S; q += kThreads) p = __dadd_rn(p, __ldcg(sp.part + (int64_t)q * m + row));
        const double sum = block_total<double>(p, red_d);
        if (threadIdx.x == 0) {
          c[row] = update_from(c[row], alpha, sum);
          sp.tickets[row] = 0u;
        }
      }
    }
  }
}

// FP64 long rows: a unit is a group of R consecutive rows times a chunk of
// the columns (the pack rows s, s + S, ... of the rows, as in the long-row
// kernel; KC is unused), so each 16-byte load of x, and each cut of an x value into
// FP32 parts for the emulated products, serves R rows; per row the first D
// of the U packs in flight go to the FP64 pipe (two chains), the rest to
// emu_fma, voted per iteration as in the long-row kernel.  A group's missing
// rows (past m) re-read row m-1 and are dropped.  Block b takes the units
// b, b + G, b + 2G, ...; with S > 1 chunks the block that finishes a
// group sums each row's S partials in chunk order (one counter per group).
template <int R, int U, int D, bool SPLIT>
__global__ void __launch_bounds__(kThreads, kRowMultiB)
    gemv_row_multi_f64_kernel(int64_t m, int64_t n, double alpha, const double* __restrict__ A, int64_t lda,
                              const double* __restrict__ x, double* __restrict__ c, const Split sp,
                              int64_t KC, int64_t units) {
  constexpr int V = 2;
  constexpr int64_t STEP = (int64_t)kThreads * V;
  constexpr int NE = (U - D) * V;  // emulated products per row per iteration
  constexpr int EFLUSH = NE > 0 && kEmuChain / NE > 0 ? kEmuChain / NE : 1;
  static_assert(D < U, "some packs are emulated");
  __shared__ double red[R][kThreads / 32];
  __shared__ int flag;

  const int S = SPLIT ? sp.S : 1;
  const int64_t PS = (int64_t)S * STEP;  // between a chunk's consecutive pack rows
  const int64_t kv1 = (n / V) * V;       // the rows' whole packs
  const int64_t jlast = (int64_t)(31 - (threadIdx.x & 31)) * V;
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {  // interleaved units
    const int64_t grp = SPLIT ? u / S : u;
    const int s = SPLIT ? (int)(u - grp * S) : 0;
    const int64_t row0 = grp * R;
    const double* Ar[R];
#pragma unroll
    for (int r = 0; r < R; ++r) Ar[r] = A + (row0 + r < m ? row0 + r : m - 1) * lda;
    double acc[R], acc2[R];
    float eh[R], el[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      acc[r] = acc2[r] = 0.0;
      eh[r] = el[r] = 0.f;
    }
    int body = 0;
    // chunk s: the pack rows s, s + S, s + 2S, ... (as in the long-row kernel)
    int64_t j = (int64_t)s * STEP + (int64_t)threadIdx.x * V;
#pragma unroll 1
    for (; j + jlast + (U - 1) * PS < kv1; j += U * PS) {
      Pack<double, V> xp[U], ap[R][U];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int q = 0; q < U; ++q) ap[r][q] = ld_stream<double, V>(Ar[r] + j + q * PS);
#pragma unroll
      for (int q = 0; q < U; ++q) xp[q] = ld_keep<double, V>(x + j + q * PS);
#pragma unroll
      for (int q = 0; q < D; ++q)
#pragma unroll
        for (int r = 0; r < R; ++r) {
          acc[r] = __fma_rn(ap[r][q].v[0], xp[q].v[0], acc[r]);
          acc2[r] = __fma_rn(ap[r][q].v[1], xp[q].v[1], acc2[r]);
        }
      unsigned rb = 0u;  // the emulated operands' ranges, OR-ed
#pragma unroll
      for (int q = D; q < U; ++q)
#pragma unroll
        for (int v = 0; v < V; ++v) {
          rb |= emu_range(xp[q].v[v]);
#pragma unroll
          for (int r = 0; r < R; ++r) rb |= emu_range(ap[r][q].v[v]);
        }
      if (__all_sync(__activemask(), rb < kEmuRange)) {
#pragma unroll
        for (int q = D; q < U; ++q)
#pragma unroll
          for (int v = 0; v < V; ++v) {
            float xh, xl;
            emu_split(xp[q].v[v], xh, xl);
#pragma unroll
            for (int r = 0; r < R; ++r) {
              float ah, al;
              emu_split(ap[r][q].v[v], ah, al);
              emu_fma(ah, al, xh, xl, eh[r], el[r]);
            }
          }
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          DPacks<NE> dp;
#pragma unroll
          for (int q = D; q < U; ++q)
#pragma unroll
            for (int v = 0; v < V; ++v) {
              dp.a[(q - D) * V + v] = ap[r][q].v[v];
              dp.x[(q - D) * V + v] = xp[q].v[v];
            }
          acc[r] = dfma_fallback(dp, acc[r]);
        }
      }
      if (++body == EFLUSH) {  // at most kEmuChain products in each FP32 pair
        body = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) emu_fold(acc[r], eh[r], el[r]);
      }
    }
#pragma unroll 1
    for (; j < kv1; j += PS) {  // remaining whole packs, one at a time
      const Pack<double, V> xq = ld_keep<double, V>(x + j);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const Pack<double, V> aq = ld_stream<double, V>(Ar[r] + j);
        acc[r] = __fma_rn(aq.v[0], xq.v[0], acc[r]);
        acc2[r] = __fma_rn(aq.v[1], xq.v[1], acc2[r]);
      }
    }
    if (s == S - 1 && kv1 + threadIdx.x < n) {  // ragged end (one column), in the last chunk
      const int64_t jj = kv1 + threadIdx.x;
      const double xj = __ldg(x + jj);
#pragma unroll
      for (int r = 0; r < R; ++r) acc[r] = __fma_rn(__ldcs(Ar[r] + jj), xj, acc[r]);
    }

    // fixed-order block sums (warp butterfly, then warps in order)
    __syncthreads();  // red is free
#pragma unroll
    for (int r = 0; r < R; ++r) {
      emu_fold(acc[r], eh[r], el[r]);
      const double v = group_sum<32>(__dadd_rn(acc[r], acc2[r]));
      if ((threadIdx.x & 31) == 0) red[r][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    const int64_t row = row0 + threadIdx.x;  // thread r < R finishes row row0 + r
    const bool mine = threadIdx.x < R && row < m;
    double t = 0.0;
    if (mine) {
#pragma unroll
      for (int w = 0; w < kThreads / 32; ++w) t = t + red[threadIdx.x][w];
    }
    if constexpr (!SPLIT) {
      if (mine) c[row] = update(c[row], alpha, t);
    } else {
      if (mine) sp.part[(int64_t)s * m + row] = t;
      multi_split_finish(sp, grp, row0, R, m, alpha, c, red[0], &flag);
    }
  }
}

// Short rows (S = 1, at most 32*8 packs).  LPR lanes per row, each with up
// to 8 packs (pack k*LPR + l of the row), so a block iteration reads
// 256/LPR consecutive rows; block b takes the row blocks b, b + G, ....
template <typename T, int V, int LPR, bool PF>
__global__ void __launch_bounds__(kThreads, PF ? kRowShortPfB : (sizeof(T) == 8 ? kRowShortB64 : 4))
    gemv_row_short_kernel(int64_t m, int64_t n, T alpha, const T* __restrict__ A, int64_t lda,
                          const T* __restrict__ x, T* __restrict__ c) {
  constexpr int GROUPS = kThreads / LPR;  // rows per block iteration
  constexpr int PMAX = 8;
  const int l = threadIdx.x % LPR;
  const int g = threadIdx.x / LPR;
  const int64_t packs = n / V;
  const int64_t kv1 = packs * V;
  const bool tail = kv1 + l < n;  // ragged end: lane l takes column kv1 + l
  const T xt = tail ? __ldg(x + kv1 + l) : T(0);
  // FP64: x is cut into FP32 parts once per block, into shared memory (NaN
  // marks a value outside the emulated range); short rows have at most 512
  // FP64 columns
  constexpr int PD = sizeof(T) == 8 ? kRowShortD64 : PMAX;  // packs on the FP64 pipe
  __shared__ float2 xs[sizeof(T) == 8 ? 256 * V : 1];
  bool xok = true;  // FP64: every x value of this lane's emulated packs is in range
  if constexpr (sizeof(T) == 8) {
    for (int64_t col = threadIdx.x; col < kv1; col += kThreads) {
      const double d = __ldg(x + col);
      float h = __int_as_float(0x7FC00000), lo = 0.f;
      if (emu_ok(d)) emu_split(d, h, lo);
      xs[col] = make_float2(h, lo);
    }
    __syncthreads();
    // a lane's columns are the same in every row, so the x half of the
    // range test is made once here
#pragma unroll
    for (int k = (sizeof(T) == 8 ? kRowShortD64 : PMAX); k < PMAX; ++k) {
      const int64_t p = (int64_t)k * LPR + l;
      if (p < packs)
#pragma unroll
        for (int v = 0; v < V; ++v) xok = xok && !isnan(xs[p * V + v].x);
    }
  }

  // every thread runs the same number of iterations (the butterfly needs
  // whole warps); rows past m are predicated off
  // this lane's packs of the row block at row b (PF: the next row block's
  // packs are loaded before the current one is summed, so loads stay in
  // flight through the arithmetic)
  const int64_t bstep = (int64_t)gridDim.x * GROUPS;
  auto load = [&](int64_t b, Pack<T, V>(&dst)[PMAX]) {
    const int64_t rw = b + g;
    if (b < m && rw < m) {
      const T* Ab = A + rw * lda;
#pragma unroll
      for (int k = 0; k < PMAX; ++k) {
        const int64_t p = (int64_t)k * LPR + l;
        if (p < packs) dst[k] = ld_stream<T, V>(Ab + p * V);
      }
    }
  };
  Pack<T, V> nxt[PMAX];
  if constexpr (PF) load(blockIdx.x * (int64_t)GROUPS, nxt);
#pragma unroll 1
  for (int64_t base = blockIdx.x * (int64_t)GROUPS; base < m; base += bstep) {
    const int64_t row = base + g;
    const bool ok = row < m;
    const T* Ar = A + (ok ? row : base) * lda;
    Pack<T, V> ap[PMAX];
    if constexpr (PF) {
#pragma unroll
      for (int k = 0; k < PMAX; ++k) ap[k] = nxt[k];
      load(base + bstep, nxt);
    } else {
      load(base, ap);
    }
    T acc = (ok && tail) ? __ldcs(Ar + kv1 + l) * xt : T(0);
    if constexpr (V > 2) {  // FP32: up to 3 ragged columns, and as few as 1 or 2 lanes per row
      if (ok)
        for (int64_t col = kv1 + l + LPR; col < n; col += LPR) acc = fma_rn(__ldcs(Ar + col), __ldg(x + col), acc);
    }
    if constexpr (sizeof(T) == 8) {
      // FP64: packs 0..PD-1 on the FP64 pipe, packs PD..7 with FP32
      // instructions (emu_fma, x cut once per block above) when every lane
      // of the warp has all of them in range; the choice is made for the
      // whole warp, so that the emulated path holds no FP64 instruction.
#pragma unroll
      for (int k = 0; k < PD; ++k) {
        const int64_t p = (int64_t)k * LPR + l;
        if (ok && p < packs) {
          const Pack<T, V> xp = ld_keep<T, V>(x + p * V);
#pragma unroll
          for (int v = 0; v < V; ++v) acc = fma_rn(ap[k].v[v], xp.v[v], acc);
        }
      }
      // packs past the row or of a row past m take no part (they add 0)
      unsigned rb = 0u;  // the emulated A operands' ranges, OR-ed (x: xok above)
#pragma unroll
      for (int k = PD; k < PMAX; ++k) {
        const int64_t p = (int64_t)k * LPR + l;
        if (ok && p < packs) {
#pragma unroll
          for (int v = 0; v < V; ++v) rb |= emu_range(ap[k].v[v]);
        }
      }
      // (a lane of a row past m votes with its x columns, which every row
      // of the warp shares: the outcome is the one of the rows inside m)
      if (__all_sync(__activemask(), rb < kEmuRange && xok)) {
        float eh = 0.f, el = 0.f;
#pragma unroll
        for (int k = PD; k < PMAX; ++k) {
          const int64_t p = (int64_t)k * LPR + l;
          if (ok && p < packs) {
#pragma unroll
            for (int v = 0; v < V; ++v) {
              float ah, al;
              emu_split(ap[k].v[v], ah, al);
              const float2 xv = xs[p * V + v];
              emu_fma(ah, al, xv.x, xv.y, eh, el);
            }
          }
        }
        emu_fold(acc, eh, el);
      } else {
        DPacks<(PMAX - PD) * V> dp;
#pragma unroll
        for (int k = PD; k < PMAX; ++k) {
          const int64_t p = (int64_t)k * LPR + l;
          const bool present = ok && p < packs;
          Pack<T, V> xq;
#pragma unroll
          for (int v = 0; v < V; ++v) xq.v[v] = T(0);
          if (present) xq = ld_keep<T, V>(x + p * V);
#pragma unroll
          for (int v = 0; v < V; ++v) {  // absent packs add 0 * 0
            dp.a[(k - PD) * V + v] = present ? (double)ap[k].v[v] : 0.0;
            dp.x[(k - PD) * V + v] = present ? (double)xq.v[v] : 0.0;
          }
        }
        acc = dfma_fallback(dp, acc);
      }
    } else {
#pragma unroll
      for (int k = 0; k < PMAX; ++k) {
        const int64_t p = (int64_t)k * LPR + l;
        if (ok && p < packs) {
          const Pack<T, V> xp = ld_keep<T, V>(x + p * V);
#pragma unroll
          for (int v = 0; v < V; ++v) acc = fma_rn(ap[k].v[v], xp.v[v], acc);
        }
      }
    }
    T sum;
    if constexpr (sizeof(T) == 4) sum = group_sum_f<LPR>(acc);
    else sum = group_sum<LPR>(acc);
    if (ok && l == 0) c[row] = update(c[row], alpha, sum);
  }
}

// Short rows off 16 bytes, x 16-byte aligned: the lane groups of the short
// kernel, with each column pack realigned from aligned packs p and p+1 of
// the row (both inside it; the row's offset MIS is per row, chosen per pack
// by selects), the first pack and the row's end element by element.  FP64
// products all on the FP64 pipe.
template <typename T, int V>
__device__ __forceinline__ T pick(const Pack<T, V>& a0, const Pack<T, V>& a1, int v, int mis) {
  const int k = v + mis;
  T r = a0.v[0];
#pragma unroll
  for (int i = 1; i < V; ++i) r = k == i ? a0.v[i] : r;
#pragma unroll
  for (int i = 0; i < V - 1; ++i) r = k == V + i ? a1.v[i] : r;
  return r;
}

template <typename T, int V, int LPR>
__global__ void __launch_bounds__(kThreads, 4)
    gemv_row_short_shift_kernel(int64_t m, int64_t n, T alpha, const T* __restrict__ A, int64_t lda,
                                const T* __restrict__ x, T* __restrict__ c) {
  constexpr int GROUPS = kThreads / LPR;
  constexpr int PMAX = 8;
  const int l = threadIdx.x % LPR;
  const int g = threadIdx.x / LPR;
#pragma unroll 1
  for (int64_t base = blockIdx.x * (int64_t)GROUPS; base < m; base += (int64_t)gridDim.x * GROUPS) {  // the same trips for every thread
    const int64_t row = base + g;
    const bool ok = row < m;
    const T* Ar = A + (ok ? row : base) * lda;
    const int mis = (int)((reinterpret_cast<uintptr_t>(Ar) / sizeof(T)) % V);
    const T* Ab = Ar - mis;
    const int64_t pv0 = mis > 0 ? 1 : 0;
    int64_t pv1 = mis > 0 ? (mis + n) / V - 1 : n / V;
    if (pv1 < pv0) pv1 = pv0;
    T acc = T(0);
#pragma unroll
    for (int k = 0; k < PMAX; ++k) {
      const int64_t p = (int64_t)k * LPR + l;
      if (ok && p >= pv0 && p < pv1) {
        const Pack<T, V> a0 = ld_stream<T, V>(Ab + p * V);
        const Pack<T, V> a1 = ld_keep<T, V>(Ab + (p + 1) * V);
        const Pack<T, V> xp = ld_keep<T, V>(x + p * V);
#pragma unroll
        for (int v = 0; v < V; ++v) acc = fma_rn(pick<T, V>(a0, a1, v, mis), xp.v[v], acc);
      }
    }
    if (ok) {
      for (int64_t col = l; col < pv0 * V && col < n; col += LPR) acc = fma_rn(__ldcs(Ar + col), __ldg(x + col), acc);
      for (int64_t col = pv1 * V + l; col < n; col += LPR) acc = fma_rn(__ldcs(Ar + col), __ldg(x + col), acc);
    }
    T sum;
    if constexpr (sizeof(T) == 4) sum = group_sum_f<LPR>(acc);
    else sum = group_sum<LPR>(acc);
    if (ok && l == 0) c[row] = update(c[row], alpha, sum);
  }
}

// Misaligned operands: warp items of RW rows (GPW = 32/LPR groups of RW rows)
// over chunks of KC columns, scalar loads.
template <typename T, int LPR, int RW>
__global__ void __launch_bounds__(kThreads, 4)
    gemv_row_scalar_kernel(int64_t m, int64_t n, T alpha, const T* __restrict__ A, int64_t lda,
                           const T* __restrict__ x, T* __restrict__ c, const Split sp, int64_t KC,
                           int64_t items) {
  constexpr int GPW = 32 / LPR;
  constexpr int ROWS = GPW * RW;
  const int S = sp.S;
  const int lane = threadIdx.x & 31;
  const int l = lane % LPR;
  const int grp = lane / LPR;
  const int64_t nwarps = (int64_t)gridDim.x * (kThreads / 32);
  for (int64_t it = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5; it < items; it += nwarps) {
    const int64_t ri = it / S;
    const int s = (int)(it - ri * S);
    const int64_t rbase = ri * ROWS;
    const int64_t row0 = rbase + (int64_t)grp * RW;
    const int64_t k0 = (int64_t)s * KC;
    const int64_t k1 = (k0 + KC < n) ? k0 + KC : n;
    double tot[RW];
    T acc[RW];
#pragma unroll
    for (int r = 0; r < RW; ++r) { tot[r] = 0.0; acc[r] = T(0); }
    int cnt = 0;
    for (int64_t j = k0 + l; j < k1; j += LPR) {
      const T xs = __ldg(x + j);
#pragma unroll
      for (int r = 0; r < RW; ++r) {
        const int64_t row = (row0 + r < m) ? row0 + r : m - 1;
        acc[r] = fma_rn(__ldcs(A + row * lda + j), xs, acc[r]);
      }
      if (++cnt == 64) {  // chains move into FP64 after 64 products
        cnt = 0;
#pragma unroll
        for (int r = 0; r < RW; ++r) { tot[r] = __dadd_rn(tot[r], (double)acc[r]); acc[r] = T(0); }
      }
    }
#pragma unroll
    for (int r = 0; r < RW; ++r) tot[r] = group_sum<LPR>(__dadd_rn(tot[r], (double)acc[r]));
    if (S == 1) {
      if (l == 0) {
#pragma unroll
        for (int r = 0; r < RW; ++r)
          if (row0 + r < m) c[row0 + r] = update_from(c[row0 + r], alpha, tot[r]);
      }
    } else {
      if (l == 0) {
#pragma unroll
        for (int r = 0; r < RW; ++r)
          if (row0 + r < m) sp.part[(int64_t)s * m + row0 + r] = tot[r];
      }
      const int rows = (int)((m - rbase < ROWS) ? m - rbase : ROWS);
      warp_split_finish<T>(sp, ri, s, rbase, rows, c, alpha);
    }
  }
}

template <typename T, int V, bool LONG>
int launch_long(const GemvArgs<T>& a, const GemvPlan& p, cudaStream_t st) {
  if constexpr (sizeof(T) == 8) {
    if (p.multi) {
      auto go = [&](auto kern) {
        const int grid = grid_size((const void*)kern, p.units, 0, kRowMultiWaves);
        kern<<<grid, kThreads, 0, st>>>(a.m, a.n, a.alpha, a.A, a.lda, a.x, a.c, p.split, p.kc, p.units);
      };
      if (p.split.S > 1) go(gemv_row_multi_f64_kernel<kRowMultiR, kRowMultiU, kRowMultiD, true>);
      else go(gemv_row_multi_f64_kernel<kRowMultiR, kRowMultiU, kRowMultiD, false>);
      return 0;
    }
  }
  // FP64 carries the FP32 emulation of half its products: more work per
  // byte, so more packs in flight per thread
  auto kern = gemv_row_long_kernel<T, V, sizeof(T) == 8 ? kRowLongU64 : kRowLongU, LONG>;
  const int grid = grid_size((const void*)kern, p.units);
  kern<<<grid, kThreads, 0, st>>>(a.m, a.n, a.alpha, a.A, a.lda, a.x, a.c, p.split, p.kc, p.units);
  return 0;
}

template <typename T, int V, int LPR>
int launch_short(const GemvArgs<T>& a, const GemvPlan& p, cudaStream_t st) {
  auto kern = gemv_row_short_kernel<T, V, LPR, (sizeof(T) == 8 ? kRowShortPf64 : kRowShortPf32)>;
  constexpr int64_t rows_per_iter = kThreads / LPR;
  const int grid = grid_size((const void*)kern, (a.m + rows_per_iter - 1) / rows_per_iter);
  kern<<<grid, kThreads, 0, st>>>(a.m, a.n, a.alpha, a.A, a.lda, a.x, a.c);
  return 0;
}

template <typename T, int LPR>
int launch_short_shift(const GemvArgs<T>& a, const GemvPlan& p, cudaStream_t st) {
  constexpr int V = 16 / sizeof(T);
  auto kern = gemv_row_short_shift_kernel<T, V, LPR>;
  constexpr int64_t rows_per_iter = kThreads / LPR;
  const int grid = grid_size((const void*)kern, (a.m + rows_per_iter - 1) / rows_per_iter);
  kern<<<grid, kThreads, 0, st>>>(a.m, a.n, a.alpha, a.A, a.lda, a.x, a.c);
  return 0;
}

template <typename T, bool LONG>
int launch_shift(const GemvArgs<T>& a, const GemvPlan& p, cudaStream_t st) {
  constexpr int V = 16 / sizeof(T);
  auto kern = gemv_row_shift_kernel<T, V, kRowLongU, LONG>;
  const int grid = grid_size((const void*)kern, p.units);
  kern<<<grid, kThreads, 0, st>>>(a.m, a.n, a.alpha, a.A, a.lda, a.x, a.c, p.split, p.kc, p.units);
  return 0;
}

template <typename T, int LPR>
int launch_scalar(const GemvArgs<T>& a, const GemvPlan& p, cudaStream_t st) {
  auto kern = gemv_row_scalar_kernel<T, LPR, kRowScalarRW>;
  const int64_t blocks = (p.units + kThreads / 32 - 1) / (kThreads / 32);
  const int grid = grid_size((const void*)kern, blocks);
  kern<<<grid, kThreads, 0, st>>>(a.m, a.n, a.alpha, a.A, a.lda, a.x, a.c, p.split, p.kc, p.units);
  return 0;
}

}  // namespace

template <typename T>
int gemv_row_launch(const GemvArgs<T>& a, const GemvPlan& p, cudaStream_t st) {
  constexpr int V = 16 / sizeof(T);
  if (p.kind == GemvPlan::kRowLong) {
    if constexpr (sizeof(T) == 4)
      return p.long_chain ? launch_long<T, V, true>(a, p, st) : launch_long<T, V, false>(a, p, st);
    else
      return launch_long<T, V, false>(a, p, st);
  }
  if (p.kind == GemvPlan::kRowShift) {
    if constexpr (sizeof(T) == 4)
      return p.long_chain ? launch_shift<T, true>(a, p, st) : launch_shift<T, false>(a, p, st);
    else
      return launch_shift<T, false>(a, p, st);
  }
  if (p.kind == GemvPlan::kRowShortShift) {
    switch (p.lpr) {
      case 32: return launch_short_shift<T, 32>(a, p, st);
      case 16: return launch_short_shift<T, 16>(a, p, st);
      case 8: return launch_short_shift<T, 8>(a, p, st);
      case 4: return launch_short_shift<T, 4>(a, p, st);
      case 2: return launch_short_shift<T, 2>(a, p, st);
      default: return launch_short_shift<T, 1>(a, p, st);
    }
  }
  if (p.kind == GemvPlan::kRowShort) {
    switch (p.lpr) {
      case 32: return launch_short<T, V, 32>(a, p, st);
      case 16: return launch_short<T, V, 16>(a, p, st);
      case 8: return launch_short<T, V, 8>(a, p, st);
      case 4: return launch_short<T, V, 4>(a, p, st);
      case 2: return launch_short<T, V, 2>(a, p, st);
      default: return launch_short<T, V, 1>(a, p, st);
    }
  }
  switch (p.lpr) {
    case 32: return launch_scalar<T, 32>(a, p, st);
    case 16: return launch_scalar<T, 16>(a, p, st);
    case 8: return launch_scalar<T, 8>(a, p, st);
    case 4: return launch_scalar<T, 4>(a, p, st);
    case 2: return launch_scalar<T, 2>(a, p, st);
    default: return launch_scalar<T, 1>(a, p, st);
  }
}

template int gemv_row_launch<float>(const GemvArgs<float>&, const GemvPlan&, cudaStream_t);
template int gemv_row_launch<double>(const GemvArgs<double>&, const GemvPlan&, cudaStream_t);

}  // namespace gb
