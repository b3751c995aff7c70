// Batched level-2 work: many independent row-major problems in ONE
// persistent launch,
//     GEMV  c_p <- c_p + alpha_p * A_p x_p   (Def. GEMV, Sec. 3.1; A FP32 or BF16)
//     GER   C_p <- C_p + alpha_p * x_p y_p^T (Def. GEM; one fma per element)
// The paper runs one GEMV at a time and notes that small problems do not
// amortise the cost of starting threads (Sec. 4.1, the speedup bound with
// its thread overhead O(t); Sec. 4.2, Analysis); on the GPU the analogue is
// a launch, and its drain, per small problem.  A host planner cuts every
// problem into tiles of whole rows of about equal cost, and each block of
// one launch streams the tiles whose cost prefix falls in its equal share
// [b*B/G, (b+1)*B/G).  The public entry points plan FP32 GEMVs; the serving
// engine plans all three kinds through the same planner.
//
// Within a tile, groups of `lpr` lanes each take one row.  GEMV: every lane
// keeps FP32 fma chains of at most 64 products folded into a compensated
// FP32 sum (TwoSum), and the group combines its lanes by a fixed butterfly;
// a row's result therefore depends only on n and the tuning entry of n's
// bucket, never on the other problems, the tile boundaries or the grid.
// GER: every element is one fma, independent of any tiling.
#include <algorithm>
#include <cstring>
#include <vector>

#include "gbblas.h"
#include "gb_common.cuh"
#include "gb_internal.h"

namespace gb {
namespace {

constexpr uint32_t kPlanMagic = 0x47425042u;  // "BPBG"
constexpr uint32_t kPlanVersion = 1u;

struct BatchHeader {  // 64 bytes
  uint32_t magic, version;
  int64_t count;       // problems
  int64_t tiles;       // T
  int64_t total_cost;  // B = prefix[T]
  int64_t off_problems, off_tiles, off_prefix;
  int64_t reserved;
};

struct BatchProblem {  // 48 bytes
  const void* A;  // GEMV: A (FP32) or its BF16 codes; GER: C (read and written)
  const float* x; // GEMV: x; GER: y (the n-vector)
  float* c;       // GEMV: c (read and written); GER: x (the m-vector, read)
  int64_t lda;    // elements
  int32_t m, n;
  float alpha;
  uint8_t vec;    // 16-byte path: matrix and n-vector 16-byte aligned, lda a multiple of a pack
  uint8_t kind;   // BatchKind
  uint16_t pad;
};

// A tile carries everything its rows need, so the kernel reads one
// descriptor per tile and never the problem table.  Fields as in
// BatchProblem, A and c moved to the tile's first row.
struct BatchTile {  // 48 bytes
  const void* A;
  const float* x;
  float* c;
  int64_t lda;
  int32_t rows, n;
  float alpha;
  uint8_t lpr_log2, u_log2, vec, kind;
};

static_assert(sizeof(BatchHeader) == 64, "plan header layout");
static_assert(sizeof(BatchProblem) == 48, "plan problem layout");
static_assert(sizeof(BatchTile) == 48, "plan tile layout");

constexpr int kTileChunk = 32;  // tile descriptors staged in shared memory at a time
constexpr int kBatchRowsGemv = 2;  // GEMV rows (16-byte path) a lane group sums at once, sharing x

// ----------------------------------------------------------------- kernel ---

__device__ __forceinline__ void fold(float& acc, float& hi, float& lo) {
  float e;
  two_sum_f(hi, acc, hi, e);
  lo = __fadd_rn(lo, e);
  acc = 0.f;
}

// A 16-byte pack of the matrix: 4 FP32 values, or 8 BF16 codes decoded
// exactly (a BF16 value is the top half of its binary32).
template <int KIND>
struct Row;

template <>
struct Row<kBatchGemvF32> {
  static constexpr int PER = 4;
  __device__ static float elem(const void* row, int e) { return __ldcs(static_cast<const float*>(row) + e); }
  __device__ static void pack(const void* row, int j, float (&v)[PER]) {
    const float4 a = __ldcs(static_cast<const float4*>(row) + j);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  }
};

template <>
struct Row<kBatchGemvBF16> {
  static constexpr int PER = 8;
  __device__ static float elem(const void* row, int e) {
    return __uint_as_float((unsigned)__ldcs(static_cast<const unsigned short*>(row) + e) << 16);
  }
  __device__ static void pack(const void* row, int j, float (&v)[PER]) {
    const uint4 a = __ldcs(static_cast<const uint4*>(row) + j);
    const unsigned w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[2 * k] = __uint_as_float(w[k] << 16);
      v[2 * k + 1] = __uint_as_float(w[k] & 0xFFFF0000u);
    }
  }
};

// One lane's part of the dot product of row r with x: packs lane, lane +
// lpr, ... (U in flight), then the ragged columns past the last whole pack.
template <int KIND, int U>
__device__ float row_dot_vec(const BatchTile& tl, int r, int lane, int lpr) {
  using R = Row<KIND>;
  constexpr int PER = R::PER;
  const void* row = static_cast<const unsigned char*>(tl.A) + (int64_t)r * tl.lda * (KIND == kBatchGemvBF16 ? 2 : 4);
  const float4* xv = reinterpret_cast<const float4*>(tl.x);
  const int P = tl.n / PER;
  float acc = 0.f, hi = 0.f, lo = 0.f;
  int cnt = 0;
  int j = lane;
#pragma unroll 1
  for (; j + (U - 1) * lpr < P; j += U * lpr) {
    float av[U][PER];
#pragma unroll
    for (int q = 0; q < U; ++q) R::pack(row, j + q * lpr, av[q]);
#pragma unroll
    for (int q = 0; q < U; ++q) {
#pragma unroll
      for (int k = 0; k < PER / 4; ++k) {
        const float4 x4 = __ldg(xv + (j + q * lpr) * (PER / 4) + k);
        acc = __fmaf_rn(av[q][4 * k + 0], x4.x, acc);
        acc = __fmaf_rn(av[q][4 * k + 1], x4.y, acc);
        acc = __fmaf_rn(av[q][4 * k + 2], x4.z, acc);
        acc = __fmaf_rn(av[q][4 * k + 3], x4.w, acc);
      }
    }
    cnt += PER * U;
    if (cnt == 64) {  // PER * U divides 64
      fold(acc, hi, lo);
      cnt = 0;
    }
  }
#pragma unroll 1
  for (; j < P; j += lpr) {
    float av[PER];
    R::pack(row, j, av);
#pragma unroll
    for (int k = 0; k < PER / 4; ++k) {
      const float4 x4 = __ldg(xv + j * (PER / 4) + k);
      acc = __fmaf_rn(av[4 * k + 0], x4.x, acc);
      acc = __fmaf_rn(av[4 * k + 1], x4.y, acc);
      acc = __fmaf_rn(av[4 * k + 2], x4.z, acc);
      acc = __fmaf_rn(av[4 * k + 3], x4.w, acc);
    }
    cnt += PER;
    if (cnt == 64) {
      fold(acc, hi, lo);
      cnt = 0;
    }
  }
  for (int e = PER * P + lane; e < tl.n; e += lpr)  // fewer than PER columns, possibly fewer lanes
    acc = __fmaf_rn(R::elem(row, e), __ldg(tl.x + e), acc);
  return __fadd_rn(hi, __fadd_rn(lo, acc));
}

// Misaligned problems: the lanes of the group stride over single elements.
template <int KIND>
__device__ float row_dot_scalar(const BatchTile& tl, int r, int lane, int lpr) {
  using R = Row<KIND>;
  const void* row = static_cast<const unsigned char*>(tl.A) + (int64_t)r * tl.lda * (KIND == kBatchGemvBF16 ? 2 : 4);
  const int n = tl.n;
  float acc = 0.f, hi = 0.f, lo = 0.f;
  int cnt = 0;
  int j = lane;
#pragma unroll 1
  for (; j + 3 * lpr < n; j += 4 * lpr) {
    float a[4], x[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) a[q] = R::elem(row, j + q * lpr);
#pragma unroll
    for (int q = 0; q < 4; ++q) x[q] = __ldg(tl.x + j + q * lpr);
#pragma unroll
    for (int q = 0; q < 4; ++q) acc = __fmaf_rn(a[q], x[q], acc);
    cnt += 4;
    if (cnt == 64) {
      fold(acc, hi, lo);
      cnt = 0;
    }
  }
#pragma unroll 1
  for (; j < n; j += lpr) acc = __fmaf_rn(R::elem(row, j), __ldg(tl.x + j), acc);
  return __fadd_rn(hi, __fadd_rn(lo, acc));
}

// GER row r: C_rj <- fma(x_r, fl(alpha * y_j), C_rj), U packs per lane in flight.
template <int U>
__device__ void row_ger_vec(const BatchTile& tl, int r, int lane, int lpr) {
  float* row = static_cast<float*>(const_cast<void*>(tl.A)) + (int64_t)r * tl.lda;
  float4* cv = reinterpret_cast<float4*>(row);
  const float4* yv = reinterpret_cast<const float4*>(tl.x);
  const float xr = tl.c[r];
  const float al = tl.alpha;
  const int P = tl.n >> 2;
  int j = lane;
#pragma unroll 1
  for (; j + (U - 1) * lpr < P; j += U * lpr) {
    float4 cc[U], yy[U];
#pragma unroll
    for (int q = 0; q < U; ++q) cc[q] = __ldcs(cv + j + q * lpr);
#pragma unroll
    for (int q = 0; q < U; ++q) yy[q] = __ldg(yv + j + q * lpr);
#pragma unroll
    for (int q = 0; q < U; ++q) {
      cc[q].x = __fmaf_rn(xr, __fmul_rn(al, yy[q].x), cc[q].x);
      cc[q].y = __fmaf_rn(xr, __fmul_rn(al, yy[q].y), cc[q].y);
      cc[q].z = __fmaf_rn(xr, __fmul_rn(al, yy[q].z), cc[q].z);
      cc[q].w = __fmaf_rn(xr, __fmul_rn(al, yy[q].w), cc[q].w);
      __stcs(cv + j + q * lpr, cc[q]);
    }
  }
#pragma unroll 1
  for (; j < P; j += lpr) {
    float4 c4 = __ldcs(cv + j);
    const float4 y4 = __ldg(yv + j);
    c4.x = __fmaf_rn(xr, __fmul_rn(al, y4.x), c4.x);
    c4.y = __fmaf_rn(xr, __fmul_rn(al, y4.y), c4.y);
    c4.z = __fmaf_rn(xr, __fmul_rn(al, y4.z), c4.z);
    c4.w = __fmaf_rn(xr, __fmul_rn(al, y4.w), c4.w);
    __stcs(cv + j, c4);
  }
  for (int e = 4 * P + lane; e < tl.n; e += lpr) row[e] = __fmaf_rn(xr, __fmul_rn(al, __ldg(tl.x + e)), row[e]);
}

__device__ void row_ger_scalar(const BatchTile& tl, int r, int lane, int lpr) {
  float* row = static_cast<float*>(const_cast<void*>(tl.A)) + (int64_t)r * tl.lda;
  const float xr = tl.c[r];
  const float al = tl.alpha;
#pragma unroll 1
  for (int j = lane; j < tl.n; j += lpr) row[j] = __fmaf_rn(xr, __fmul_rn(al, __ldg(tl.x + j)), row[j]);
}

// Rows r, r + step, ... (R of them, the first nr valid; the others re-read
// row r and are dropped) of an FP32 or BF16 GEMV tile: each float4 of x
// serves all R rows (with two bytes per element, a lone BF16 row would read
// twice its own bytes of x).  Every row takes exactly the steps of a lone row
// (same packs per lane, same chain folds), so its result does not depend on
// its neighbours.
template <int KIND>
__device__ __forceinline__ void decode4(const uint4& q, int h, float (&f)[4]) {
  if constexpr (KIND == kBatchGemvBF16) {
    const unsigned w0 = h ? q.z : q.x, w1 = h ? q.w : q.y;
    f[0] = __uint_as_float(w0 << 16);
    f[1] = __uint_as_float(w0 & 0xFFFF0000u);
    f[2] = __uint_as_float(w1 << 16);
    f[3] = __uint_as_float(w1 & 0xFFFF0000u);
  } else {
    f[0] = __uint_as_float(q.x);
    f[1] = __uint_as_float(q.y);
    f[2] = __uint_as_float(q.z);
    f[3] = __uint_as_float(q.w);
  }
}

template <int KIND, int U, int R>
__device__ void rows_dot(const BatchTile& tl, int r, int step, int nr, int lane, int lpr, float (&out)[R]) {
  constexpr int EB = KIND == kBatchGemvBF16 ? 2 : 4;
  constexpr int PER = 16 / EB;   // elements per 16-byte pack
  constexpr int H = PER / 4;     // float4s of x per pack
  const int P = tl.n / PER;
  const uint4* rowp[R];
#pragma unroll
  for (int k = 0; k < R; ++k)
    rowp[k] = reinterpret_cast<const uint4*>(static_cast<const unsigned char*>(tl.A) +
                                             (int64_t)(k < nr ? r + k * step : r) * tl.lda * EB);
  const float4* xv = reinterpret_cast<const float4*>(tl.x);
  float acc[R], hi[R], lo[R];
#pragma unroll
  for (int k = 0; k < R; ++k) acc[k] = hi[k] = lo[k] = 0.f;
  int cnt = 0;
  int j = lane;
#pragma unroll 1
  for (; j + (U - 1) * lpr < P; j += U * lpr) {
    uint4 q[U][R];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int k = 0; k < R; ++k) q[u][k] = __ldcs(rowp[k] + j + u * lpr);
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int h = 0; h < H; ++h) {
        const float4 x4 = __ldg(xv + (j + u * lpr) * H + h);
#pragma unroll
        for (int k = 0; k < R; ++k) {
          float f[4];
          decode4<KIND>(q[u][k], h, f);
          acc[k] = __fmaf_rn(f[0], x4.x, acc[k]);
          acc[k] = __fmaf_rn(f[1], x4.y, acc[k]);
          acc[k] = __fmaf_rn(f[2], x4.z, acc[k]);
          acc[k] = __fmaf_rn(f[3], x4.w, acc[k]);
        }
      }
    cnt += PER * U;
    if (cnt == 64) {  // PER * U divides 64
#pragma unroll
      for (int k = 0; k < R; ++k) fold(acc[k], hi[k], lo[k]);
      cnt = 0;
    }
  }
#pragma unroll 1
  for (; j < P; j += lpr) {
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const float4 x4 = __ldg(xv + j * H + h);
#pragma unroll
      for (int k = 0; k < R; ++k) {
        float f[4];
        decode4<KIND>(__ldcs(rowp[k] + j), h, f);
        acc[k] = __fmaf_rn(f[0], x4.x, acc[k]);
        acc[k] = __fmaf_rn(f[1], x4.y, acc[k]);
        acc[k] = __fmaf_rn(f[2], x4.z, acc[k]);
        acc[k] = __fmaf_rn(f[3], x4.w, acc[k]);
      }
    }
    cnt += PER;
    if (cnt == 64) {
#pragma unroll
      for (int k = 0; k < R; ++k) fold(acc[k], hi[k], lo[k]);
      cnt = 0;
    }
  }
  for (int e = PER * P + lane; e < tl.n; e += lpr) {  // fewer than PER columns, possibly fewer lanes
    const float xe = __ldg(tl.x + e);
#pragma unroll
    for (int k = 0; k < R; ++k)
      acc[k] = __fmaf_rn(Row<KIND>::elem(rowp[k], e), xe, acc[k]);
  }
#pragma unroll
  for (int k = 0; k < R; ++k) out[k] = __fadd_rn(hi[k], __fadd_rn(lo[k], acc[k]));
}

template <int KIND, int R>
__device__ __forceinline__ void rows_dot_u(const BatchTile& tl, int r, int step, int nr, int lane, int lpr,
                                           float (&out)[R]) {
  switch (tl.u_log2) {
    case 0: rows_dot<KIND, 1, R>(tl, r, step, nr, lane, lpr, out); break;
    case 1: rows_dot<KIND, 2, R>(tl, r, step, nr, lane, lpr, out); break;
    default: rows_dot<KIND, 4, R>(tl, r, step, nr, lane, lpr, out); break;
  }
}

template <int KIND>
__device__ __forceinline__ float row_dot(const BatchTile& tl, int r, int lane, int lpr) {
  if (!tl.vec) return row_dot_scalar<KIND>(tl, r, lane, lpr);
  switch (tl.u_log2) {
    case 0: return row_dot_vec<KIND, 1>(tl, r, lane, lpr);
    case 1: return row_dot_vec<KIND, 2>(tl, r, lane, lpr);
    default: return row_dot_vec<KIND, 4>(tl, r, lane, lpr);
  }
}

__device__ __forceinline__ void row_ger(const BatchTile& tl, int r, int lane, int lpr) {
  if (!tl.vec) return row_ger_scalar(tl, r, lane, lpr);
  switch (tl.u_log2) {
    case 0: return row_ger_vec<1>(tl, r, lane, lpr);
    case 1: return row_ger_vec<2>(tl, r, lane, lpr);
    default: return row_ger_vec<4>(tl, r, lane, lpr);
  }
}

// One step of the compensated dot product Dot2 (Ogita, Rump & Oishi, 2005)
// in FP32: (p, s) <- p + s + a*b with the product split exactly by an fma
// (TwoProduct) and the sum by Knuth's TwoSum.
__device__ __forceinline__ void dot2_step(float a, float b, float& p, float& s) {
  const float h = __fmul_rn(a, b);
  const float r = __fmaf_rn(a, b, -h);
  float q;
  two_sum_f(p, h, p, q);
  s = __fadd_rn(s, __fadd_rn(q, r));
}

// This thread's part of a DOT tile (A . x over n elements): elements (or
// 16-byte packs) t, t + 256, ... in two Dot2 chains, returned in FP64.
__device__ double dot2_part(const BatchTile& tl) {
  const float* a = static_cast<const float*>(tl.A);
  const float* b = tl.x;
  const int n = tl.n;
  float p0 = 0.f, s0 = 0.f, p1 = 0.f, s1 = 0.f;
  int e0 = 0;
  if (tl.vec) {
    const float4* a4 = reinterpret_cast<const float4*>(a);
    const float4* b4 = reinterpret_cast<const float4*>(b);
    const int P = n >> 2;
    int j = threadIdx.x;
#pragma unroll 1
    for (; j + kThreads < P; j += 2 * kThreads) {  // two packs of each vector in flight
      const float4 x0 = __ldcs(a4 + j), y0 = __ldcs(b4 + j);
      const float4 x1 = __ldcs(a4 + j + kThreads), y1 = __ldcs(b4 + j + kThreads);
      dot2_step(x0.x, y0.x, p0, s0);
      dot2_step(x0.y, y0.y, p1, s1);
      dot2_step(x0.z, y0.z, p0, s0);
      dot2_step(x0.w, y0.w, p1, s1);
      dot2_step(x1.x, y1.x, p0, s0);
      dot2_step(x1.y, y1.y, p1, s1);
      dot2_step(x1.z, y1.z, p0, s0);
      dot2_step(x1.w, y1.w, p1, s1);
    }
    if (j < P) {
      const float4 x0 = __ldcs(a4 + j), y0 = __ldcs(b4 + j);
      dot2_step(x0.x, y0.x, p0, s0);
      dot2_step(x0.y, y0.y, p1, s1);
      dot2_step(x0.z, y0.z, p0, s0);
      dot2_step(x0.w, y0.w, p1, s1);
    }
    e0 = 4 * P;
  }
  for (int e = e0 + threadIdx.x; e < n; e += kThreads) dot2_step(__ldcs(a + e), __ldcs(b + e), p0, s0);
  return __dadd_rn(__dadd_rn((double)p0, (double)s0), __dadd_rn((double)p1, (double)s1));
}

// First t in [0, T] with prefix[t] >= v (prefix[0] = 0, prefix[T] = B).
__device__ __forceinline__ int64_t first_at_least(const int64_t* prefix, int64_t T, int64_t v) {
  int64_t lo = 0, hi = T;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (__ldg(prefix + mid) < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Copy tiles [t, t + k) of the plan into shared memory (16 bytes per lane).
__device__ __forceinline__ void stage_tiles(BatchTile* dst, const BatchTile* src, int k) {
  constexpr int kWords = (int)sizeof(BatchTile) / 16;
  for (int i = threadIdx.x; i < k * kWords; i += kThreads)
    cp_async_cg16(smem_u32(reinterpret_cast<const unsigned char*>(dst) + 16 * i),
                  reinterpret_cast<const unsigned char*>(src) + 16 * i);
  cp_async_commit();
}

__global__ void __launch_bounds__(kThreads, 3) gemv_batch_kernel(const unsigned char* __restrict__ plan) {
  __shared__ __align__(16) BatchTile stage[2][kTileChunk];
  __shared__ double red[kThreads / 32];
  const BatchHeader* h = reinterpret_cast<const BatchHeader*>(plan);
  const int64_t T = h->tiles, B = h->total_cost;
  const BatchTile* tiles = reinterpret_cast<const BatchTile*>(plan + h->off_tiles);
  const int64_t* prefix = reinterpret_cast<const int64_t*>(plan + h->off_prefix);
  const int64_t G = gridDim.x;
  const int64_t t0 = first_at_least(prefix, T, B * (int64_t)blockIdx.x / G);
  const int64_t t1 = first_at_least(prefix, T, B * ((int64_t)blockIdx.x + 1) / G);
  if (t0 >= t1) return;  // uniform over the block

  // Tile descriptors arrive in chunks, the next chunk's copy in flight while
  // the current one is processed.
  auto chunk = [&](int64_t from) { return t1 - from < kTileChunk ? (int)(t1 - from) : kTileChunk; };
  stage_tiles(stage[0], tiles + t0, chunk(t0));
  int buf = 0;
  for (int64_t c0 = t0; c0 < t1; c0 += kTileChunk, buf ^= 1) {
    const int k = chunk(c0);
    if (c0 + kTileChunk < t1) {
      stage_tiles(stage[buf ^ 1], tiles + c0 + kTileChunk, chunk(c0 + kTileChunk));
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();  // the current chunk is visible to every lane
    for (int i = 0; i < k; ++i) {
      const BatchTile pb = stage[buf][i];
      const int lg = pb.lpr_log2;
      const int lpr = 1 << lg;
      const int lane = threadIdx.x & (lpr - 1);
      const int wl = threadIdx.x & 31;
      // the lanes of this thread's group (aligned run of lpr lanes of the warp)
      const unsigned mask = lpr == 32 ? 0xffffffffu : ((1u << lpr) - 1u) << (wl & ~(lpr - 1));
      const int groups = kThreads >> lg;
      if (pb.kind == kBatchDotF32) {  // the whole block, the final sum in FP64 (uniform over the block)
        const double v = block_sum(dot2_part(pb), red);
        if (threadIdx.x == 0) pb.c[0] = (float)__dadd_rn((double)pb.c[0], v);
        continue;
      }
      if (pb.kind != kBatchGerF32 && pb.vec) {  // kBatchRowsGemv rows at a time
        constexpr int RB = kBatchRowsGemv;
        for (int r = threadIdx.x >> lg; r < pb.rows; r += RB * groups) {  // uniform over the group
          const int nr = min(RB, (pb.rows - r + groups - 1) / groups);
          float v[RB];
          if (pb.kind == kBatchGemvBF16) rows_dot_u<kBatchGemvBF16, RB>(pb, r, groups, nr, lane, lpr, v);
          else rows_dot_u<kBatchGemvF32, RB>(pb, r, groups, nr, lane, lpr, v);
#pragma unroll
          for (int k = 0; k < RB; ++k) {
            for (int o = lpr >> 1; o > 0; o >>= 1) v[k] = __fadd_rn(v[k], __shfl_xor_sync(mask, v[k], o));
            if (lane == 0 && k < nr) pb.c[r + k * groups] = __fmaf_rn(pb.alpha, v[k], pb.c[r + k * groups]);
          }
        }
        continue;
      }
      for (int r = threadIdx.x >> lg; r < pb.rows; r += groups) {  // uniform over the group
        if (pb.kind == kBatchGerF32) {
          row_ger(pb, r, lane, lpr);
          continue;
        }
        float v = pb.kind == kBatchGemvBF16 ? row_dot<kBatchGemvBF16>(pb, r, lane, lpr)
                                            : row_dot<kBatchGemvF32>(pb, r, lane, lpr);
        for (int o = lpr >> 1; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(mask, v, o));
        if (lane == 0) pb.c[r] = __fmaf_rn(pb.alpha, v, pb.c[r]);
      }
    }
    __syncthreads();  // every lane is done with this buffer before it is refilled
  }
}

// ---------------------------------------------------------------- planner ---

constexpr int64_t kTileOverhead = 256;  // cost units charged per tile (descriptor, x, tail)

inline int bucket_of(int64_t n) {
  int b = 0;
  while (b < GB_BATCH_BUCKETS - 1 && (int64_t(1) << b) < n) ++b;
  return b;
}

inline int log2_exact(int v) {
  if (v <= 0 || v > 64) return -1;
  int l = 0;
  while ((1 << l) < v) ++l;
  return (1 << l) == v ? l : -1;
}

inline bool tuning_ok(const gb_batch_tuning& t) {
  const int l = log2_exact(t.lanes_per_row);
  const int u = log2_exact(t.packs_per_iter);
  return l >= 0 && l <= 5 && u >= 0 && u <= 2 && t.tile_bytes >= 4096 && t.reserved == 0;
}

inline int elem_bytes(int kind) { return kind == kBatchGemvBF16 ? 2 : 4; }

// The tuning entry follows the row's length in 4-byte words: a BF16 row of
// n elements takes the entry of an FP32 row of ceil(n / 2).
inline int bucket_of_item(const BatchItem& it) {
  return bucket_of(it.kind == kBatchGemvBF16 ? (it.n + 1) / 2 : it.n);
}

// Rows per tile: about tile_bytes of the matrix, a multiple of the block's
// row groups (256 / lpr), at least one group.
inline int64_t tile_rows(const BatchItem& it, const gb_batch_tuning& t) {
  // GEMV lane groups take kBatchRowsGemv rows at a time
  const int64_t groups = kThreads / t.lanes_per_row * (it.kind == kBatchGerF32 ? 1 : kBatchRowsGemv);
  const int64_t row_bytes = elem_bytes(it.kind) * (it.n > 0 ? it.n : 1);
  int64_t r = (int64_t)t.tile_bytes / row_bytes;
  r = r / groups * groups;
  return r < groups ? groups : r;
}

// Cost units of a tile: bytes it moves (GER reads and writes its rows).
inline int64_t tile_cost(const BatchItem& it, int64_t rows) {
  const int64_t row = it.kind == kBatchGerF32 ? 8 * it.n : elem_bytes(it.kind) * it.n;
  return rows * (row + 8) + 4 * it.n + kTileOverhead;
}

inline bool active(const BatchItem& it) { return it.m > 0 && it.n > 0 && it.alpha != 0.f; }

inline bool shape_ok(const BatchItem& it) {
  return it.m >= 0 && it.n >= 0 && it.m <= INT32_MAX && it.n <= INT32_MAX && it.reserved == 0 &&
         it.reserved2 == 0 &&
         (it.kind == kBatchGemvF32 || it.kind == kBatchGemvBF16 || it.kind == kBatchGerF32 ||
          (it.kind == kBatchDotF32 && it.m <= 1 && (it.alpha == 1.f || it.alpha == 0.f)));
}

inline int64_t count_tiles(int64_t count, const BatchItem* items, const gb_batch_tuning* table) {
  int64_t T = 0;
  for (int64_t p = 0; p < count; ++p) {
    if (!active(items[p])) continue;
    const int64_t R = tile_rows(items[p], table[bucket_of_item(items[p])]);
    T += (items[p].m + R - 1) / R;
  }
  return T;
}

inline int64_t align16(int64_t v) { return (v + 15) / 16 * 16; }

struct Layout {
  int64_t problems, tiles, prefix, total;
};

inline Layout layout_of(int64_t count, int64_t T) {
  Layout L;
  L.problems = (int64_t)sizeof(BatchHeader);
  L.tiles = align16(L.problems + count * (int64_t)sizeof(BatchProblem));
  L.prefix = align16(L.tiles + T * (int64_t)sizeof(BatchTile));
  L.total = align16(L.prefix + (T + 1) * (int64_t)sizeof(int64_t));
  return L;
}

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

struct Interval {
  uintptr_t lo, hi;  // [lo, hi)
};

// Some interval of `a` meets some interval of `b` (both lists sorted by lo;
// `a` pairwise disjoint).
bool meets(const std::vector<Interval>& a, const std::vector<Interval>& b) {
  for (const Interval& v : b) {
    // first interval of a whose hi > v.lo
    auto it = std::upper_bound(a.begin(), a.end(), v.lo,
                               [](uintptr_t x, const Interval& w) { return x < w.hi; });
    if (it != a.end() && it->lo < v.hi) return true;
  }
  return false;
}

}  // namespace

size_t batch_plan_bytes(int64_t count, const BatchItem* items, const gb_batch_tuning* table) {
  if (count < 0 || (count > 0 && !items)) return 0;
  gb_batch_tuning def[GB_BATCH_BUCKETS];
  if (!table) {
    gb_sgemv_batch_default_tuning(def);
    table = def;
  }
  for (int b = 0; b < GB_BATCH_BUCKETS; ++b)
    if (!tuning_ok(table[b])) return 0;
  for (int64_t p = 0; p < count; ++p)
    if (!shape_ok(items[p])) return 0;
  return (size_t)layout_of(count, count_tiles(count, items, table)).total;
}

int batch_plan(int64_t count, const BatchItem* items, const gb_batch_tuning* table, void* plan,
               size_t plan_bytes) {
  if (count < 0) return -1;
  gb_batch_tuning def[GB_BATCH_BUCKETS];
  if (!table) {
    gb_sgemv_batch_default_tuning(def);
    table = def;
  }
  for (int b = 0; b < GB_BATCH_BUCKETS; ++b)
    if (!tuning_ok(table[b])) return -9;
  std::vector<Interval> outs, ins;
  for (int64_t p = 0; p < count; ++p) {
    const BatchItem& it = items[p];
    if (it.m < 0 || it.m > INT32_MAX) return -2;
    if (!shape_ok(it)) return -3;
    if (it.lda < (it.n > 1 ? it.n : 1)) return -4;
    if (!active(it)) continue;
    if (!it.A) return -6;
    if (!it.x) return -7;
    if (!it.c) return -8;
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(it.A);
    const uintptr_t x0 = reinterpret_cast<uintptr_t>(it.x);
    const uintptr_t c0 = reinterpret_cast<uintptr_t>(it.c);
    const unsigned __int128 ab =
        ((unsigned __int128)(it.m - 1) * (uint64_t)it.lda + (uint64_t)it.n) * (unsigned)elem_bytes(it.kind);
    if (ab > (unsigned __int128)(UINTPTR_MAX - a0)) return -4;  // the matrix would run past the address space
    const Interval a{a0, a0 + (uintptr_t)ab}, x{x0, x0 + (uintptr_t)(it.n * 4)}, c{c0, c0 + (uintptr_t)(it.m * 4)};
    if (it.kind == kBatchGerF32) {  // writes C, reads x and y
      outs.push_back(a);
      ins.push_back(x);
      ins.push_back(c);
    } else {                        // writes c, reads A and x
      outs.push_back(c);
      ins.push_back(a);
      ins.push_back(x);
    }
  }
  auto by_lo = [](const Interval& a, const Interval& b) { return a.lo < b.lo; };
  std::sort(outs.begin(), outs.end(), by_lo);
  for (size_t i = 1; i < outs.size(); ++i)
    if (outs[i].lo < outs[i - 1].hi) return -8;  // two problems write the same memory
  std::sort(ins.begin(), ins.end(), by_lo);
  if (meets(outs, ins)) return -8;               // an output overlaps some input
  if (!plan || !aligned16(plan)) return -10;

  const int64_t T = count_tiles(count, items, table);
  const Layout L = layout_of(count, T);
  if (plan_bytes < (size_t)L.total) return -11;
  unsigned char* base = static_cast<unsigned char*>(plan);
  std::memset(base, 0, (size_t)L.total);
  BatchHeader* h = reinterpret_cast<BatchHeader*>(base);
  BatchProblem* probs = reinterpret_cast<BatchProblem*>(base + L.problems);
  BatchTile* tiles = reinterpret_cast<BatchTile*>(base + L.tiles);
  int64_t* prefix = reinterpret_cast<int64_t*>(base + L.prefix);
  int64_t t = 0, cost = 0;
  for (int64_t p = 0; p < count; ++p) {
    const BatchItem& it = items[p];
    const int eb = elem_bytes(it.kind);
    BatchProblem& pb = probs[p];
    pb.A = it.A;
    pb.x = it.x;
    pb.c = it.c;
    pb.lda = it.lda;
    pb.m = (int32_t)it.m;
    pb.n = (int32_t)it.n;
    pb.alpha = it.alpha;
    pb.kind = (uint8_t)it.kind;
    pb.vec = aligned16(it.A) && aligned16(it.x) && (it.kind == kBatchDotF32 || (it.lda * eb) % 16 == 0);
    if (!active(it)) continue;
    const gb_batch_tuning& tu = table[bucket_of_item(it)];
    const int64_t R = tile_rows(it, tu);
    for (int64_t r0 = 0; r0 < it.m; r0 += R) {
      BatchTile& tl = tiles[t];
      tl.A = static_cast<const unsigned char*>(it.A) + r0 * it.lda * eb;
      tl.x = it.x;
      tl.c = it.c + r0;
      tl.lda = it.lda;
      tl.rows = (int32_t)std::min<int64_t>(R, it.m - r0);
      tl.n = (int32_t)it.n;
      tl.alpha = it.alpha;
      tl.lpr_log2 = (uint8_t)log2_exact(tu.lanes_per_row);
      tl.u_log2 = (uint8_t)log2_exact(tu.packs_per_iter);
      tl.vec = pb.vec;
      tl.kind = pb.kind;
      prefix[t] = cost;
      cost += tile_cost(it, tl.rows);
      ++t;
    }
  }
  prefix[T] = cost;
  h->magic = kPlanMagic;
  h->version = kPlanVersion;
  h->count = count;
  h->tiles = T;
  h->total_cost = cost;
  h->off_problems = L.problems;
  h->off_tiles = L.tiles;
  h->off_prefix = L.prefix;
  return GB_OK;
}

}  // namespace gb

// ------------------------------------------------------------------ C ABI ---

using namespace gb;

namespace {

// FP32 GEMV problems of the public entry points as batch items.
std::vector<BatchItem> sgemv_items(int64_t count, const int64_t* m, const int64_t* n, const int64_t* lda,
                                   const float* alpha, const float* const* A, const float* const* x,
                                   float* const* c) {
  std::vector<BatchItem> items((size_t)count);
  for (int64_t p = 0; p < count; ++p) {
    BatchItem& it = items[(size_t)p];
    it = BatchItem{};
    it.kind = kBatchGemvF32;
    it.m = m[p];
    it.n = n[p];
    it.lda = lda ? lda[p] : (n[p] > 1 ? n[p] : 1);
    it.alpha = alpha ? alpha[p] : 1.f;
    it.A = A ? const_cast<float*>(A[p]) : nullptr;
    it.x = x ? x[p] : nullptr;
    it.c = c ? c[p] : nullptr;
  }
  return items;
}

}  // namespace

extern "C" {

void gb_sgemv_batch_default_tuning(gb_batch_tuning* table) {
  if (!table) return;
  for (int b = 0; b < GB_BATCH_BUCKETS; ++b) {
    const int64_t packs = b >= 2 ? (int64_t(1) << (b - 2)) : 1;  // at the bucket's largest n
    int lpr = 8;
    while (lpr < 32 && packs / lpr > 4) lpr <<= 1;  // about 4 packs per lane, up to 32 lanes
    int u = 1;
    while (u < 4 && packs / lpr >= 2 * u) u <<= 1;
    table[b] = gb_batch_tuning{lpr, u, 256 << 10, 0};
  }
}

size_t gb_sgemv_batch_plan_bytes(int64_t count, const int64_t* m, const int64_t* n, const float* alpha,
                                 const gb_batch_tuning* table) {
  if (count < 0 || (count > 0 && (!m || !n))) return 0;
  const std::vector<BatchItem> items = sgemv_items(count, m, n, nullptr, alpha, nullptr, nullptr, nullptr);
  return batch_plan_bytes(count, items.data(), table);
}

int gb_sgemv_batch_plan(int64_t count, const int64_t* m, const int64_t* n, const int64_t* lda,
                        const float* alpha, const float* const* A, const float* const* x,
                        float* const* c, const gb_batch_tuning* table, void* plan, size_t plan_bytes) {
  if (count < 0) return -1;
  if (count > 0 && (!m || !n || !lda || !alpha || !A || !x || !c)) {
    if (!m) return -2;
    if (!n) return -3;
    if (!lda) return -4;
    if (!alpha) return -5;
    if (!A) return -6;
    if (!x) return -7;
    return -8;
  }
  for (int64_t p = 0; p < count; ++p) {  // m is checked before n, as the argument order goes
    if (m[p] < 0 || m[p] > INT32_MAX) return -2;
    if (n[p] < 0 || n[p] > INT32_MAX) return -3;
  }
  const std::vector<BatchItem> items = sgemv_items(count, m, n, lda, alpha, A, x, c);
  return batch_plan(count, items.data(), table, plan, plan_bytes);
}

size_t gb_batch_plan_bytes(int64_t count, const gb_batch_item* items, const gb_batch_tuning* table) {
  return batch_plan_bytes(count, items, table);
}

int gb_batch_plan(int64_t count, const gb_batch_item* items, const gb_batch_tuning* table, void* plan,
                  size_t plan_bytes) {
  if (count < 0) return -1;
  if (count > 0 && !items) return -2;
  const int st = batch_plan(count, items, table, plan, plan_bytes);
  if (st >= 0) return st;
  if (st == -9) return -3;
  if (st == -10) return -4;
  if (st == -11) return -5;
  return -2;
}

int gb_sgemv_batch(const void* plan_host, const void* plan_dev, gb_stream stream) {
  const BatchHeader* h = static_cast<const BatchHeader*>(plan_host);
  if (!h || h->magic != kPlanMagic || h->version != kPlanVersion) return -1;
  if (!plan_dev || !aligned16(plan_dev)) return -2;
  if (h->tiles == 0) return GB_OK;
  const int blocks = grid_size((const void*)gemv_batch_kernel, h->tiles);
  gemv_batch_kernel<<<blocks, kThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<const unsigned char*>(plan_dev));
  return cudaPeekAtLastError() == cudaSuccess ? GB_OK : GB_ERR_CUDA;
}

int64_t gb_sgemv_batch_tiles(const void* plan_host) {
  const BatchHeader* h = static_cast<const BatchHeader*>(plan_host);
  if (!h || h->magic != kPlanMagic || h->version != kPlanVersion) return -1;
  return h->tiles;
}

}  // extern "C"
