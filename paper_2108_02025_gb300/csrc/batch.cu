// Batched FP32 GEMV: many independent row-major problems
//     c_p <- c_p + alpha_p * A_p x_p          (Def. GEMV, Sec. 3.1, per problem)
// in ONE persistent launch.  The paper runs one GEMV at a time and notes that
// small problems do not amortise the cost of starting threads (Sec. 4.1, the
// speedup bound with its thread overhead O(t); Sec. 4.2, Analysis); on the
// GPU the analogue is a launch, and its drain, per small GEMV.  Here a host
// planner cuts every problem into tiles of whole rows of about equal bytes,
// and each block of one launch streams the tiles whose cost prefix falls in
// its equal share [b*B/G, (b+1)*B/G).
//
// Within a tile, groups of `lpr` lanes each sum one row: every lane keeps
// FP32 fma chains of at most 64 products folded into a compensated FP32 sum
// (TwoSum), and the group combines its lanes by a fixed butterfly.  A row's
// result therefore depends only on n and the tuning entry of n's bucket,
// never on the other problems, the tile boundaries or the grid.
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
  const float* A;
  const float* x;
  float* c;
  int64_t lda;
  int32_t m, n;
  float alpha;
  int32_t vec;  // A, x 16-byte aligned and lda a multiple of 4
};

// A tile carries everything its rows need, so the kernel reads one
// descriptor per tile and never the problem table.
struct BatchTile {  // 48 bytes
  const float* A;  // first row of the tile
  const float* x;
  float* c;        // output of the first row
  int64_t lda;
  int32_t rows, n;
  float alpha;
  uint8_t lpr_log2, u_log2, vec, pad;
};

static_assert(sizeof(BatchHeader) == 64, "plan header layout");
static_assert(sizeof(BatchProblem) == 48, "plan problem layout");
static_assert(sizeof(BatchTile) == 48, "plan tile layout");

constexpr int kTileChunk = 32;  // tile descriptors staged in shared memory at a time

// ----------------------------------------------------------------- kernel ---

__device__ __forceinline__ void fold(float& acc, float& hi, float& lo) {
  float e;
  two_sum_f(hi, acc, hi, e);
  lo = __fadd_rn(lo, e);
  acc = 0.f;
}

__device__ __forceinline__ void fma4(float& acc, const float4& a, const float4& x) {
  acc = __fmaf_rn(a.x, x.x, acc);
  acc = __fmaf_rn(a.y, x.y, acc);
  acc = __fmaf_rn(a.z, x.z, acc);
  acc = __fmaf_rn(a.w, x.w, acc);
}

// One lane's part of row `row`: packs lane, lane + lpr, ... (U in flight),
// then the ragged columns past the last whole pack.
template <int U>
__device__ float row_vec(const BatchTile& pb, int r, int lane, int lpr) {
  const float* Ar = pb.A + (int64_t)r * pb.lda;
  const float4* a = reinterpret_cast<const float4*>(Ar);
  const float4* xv = reinterpret_cast<const float4*>(pb.x);
  const int P = pb.n >> 2;
  float acc = 0.f, hi = 0.f, lo = 0.f;
  int cnt = 0;
  int j = lane;
#pragma unroll 1
  for (; j + (U - 1) * lpr < P; j += U * lpr) {
    float4 av[U], xx[U];
#pragma unroll
    for (int q = 0; q < U; ++q) av[q] = __ldcs(a + j + q * lpr);
#pragma unroll
    for (int q = 0; q < U; ++q) xx[q] = __ldg(xv + j + q * lpr);
#pragma unroll
    for (int q = 0; q < U; ++q) fma4(acc, av[q], xx[q]);
    cnt += 4 * U;
    if (cnt == 64) {  // 4U divides 64
      fold(acc, hi, lo);
      cnt = 0;
    }
  }
#pragma unroll 1
  for (; j < P; j += lpr) {
    fma4(acc, __ldcs(a + j), __ldg(xv + j));
    cnt += 4;
    if (cnt == 64) {
      fold(acc, hi, lo);
      cnt = 0;
    }
  }
  for (int e = 4 * P + lane; e < pb.n; e += lpr)  // at most 3 columns, fewer lanes possible
    acc = __fmaf_rn(__ldcs(Ar + e), __ldg(pb.x + e), acc);
  return __fadd_rn(hi, __fadd_rn(lo, acc));
}

// Misaligned problems: the lanes of the group stride over single elements.
__device__ float row_scalar(const BatchTile& pb, int r, int lane, int lpr) {
  const float* Ar = pb.A + (int64_t)r * pb.lda;
  const int n = pb.n;
  float acc = 0.f, hi = 0.f, lo = 0.f;
  int cnt = 0;
  int j = lane;
#pragma unroll 1
  for (; j + 3 * lpr < n; j += 4 * lpr) {
    float a[4], x[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) a[q] = __ldcs(Ar + j + q * lpr);
#pragma unroll
    for (int q = 0; q < 4; ++q) x[q] = __ldg(pb.x + j + q * lpr);
#pragma unroll
    for (int q = 0; q < 4; ++q) acc = __fmaf_rn(a[q], x[q], acc);
    cnt += 4;
    if (cnt == 64) {
      fold(acc, hi, lo);
      cnt = 0;
    }
  }
#pragma unroll 1
  for (; j < n; j += lpr) acc = __fmaf_rn(__ldcs(Ar + j), __ldg(pb.x + j), acc);
  return __fadd_rn(hi, __fadd_rn(lo, acc));
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
      for (int r = threadIdx.x >> lg; r < pb.rows; r += kThreads >> lg) {  // uniform over the group
        float v;
        if (pb.vec) {
          switch (pb.u_log2) {
            case 0: v = row_vec<1>(pb, r, lane, lpr); break;
            case 1: v = row_vec<2>(pb, r, lane, lpr); break;
            default: v = row_vec<4>(pb, r, lane, lpr); break;
          }
        } else {
          v = row_scalar(pb, r, lane, lpr);
        }
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

// Rows per tile for a problem of n columns: about tile_bytes of A, a
// multiple of the block's row groups (256 / lpr), at least one group each.
inline int64_t tile_rows(int64_t n, const gb_batch_tuning& t) {
  const int64_t groups = kThreads / t.lanes_per_row;
  const int64_t row_bytes = 4 * (n > 0 ? n : 1);
  int64_t r = (int64_t)t.tile_bytes / row_bytes;
  r = r / groups * groups;
  return r < groups ? groups : r;
}

inline bool active(int64_t m, int64_t n, float alpha) { return m > 0 && n > 0 && alpha != 0.f; }

inline int64_t count_tiles(int64_t count, const int64_t* m, const int64_t* n, const float* alpha,
                           const gb_batch_tuning* table) {
  int64_t T = 0;
  for (int64_t p = 0; p < count; ++p) {
    if (!active(m[p], n[p], alpha ? alpha[p] : 1.f)) continue;
    const int64_t R = tile_rows(n[p], table[bucket_of(n[p])]);
    T += (m[p] + R - 1) / R;
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
}  // namespace gb

// ------------------------------------------------------------------ C ABI ---

using namespace gb;

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
  gb_batch_tuning def[GB_BATCH_BUCKETS];
  if (!table) {
    gb_sgemv_batch_default_tuning(def);
    table = def;
  }
  for (int b = 0; b < GB_BATCH_BUCKETS; ++b)
    if (!tuning_ok(table[b])) return 0;
  for (int64_t p = 0; p < count; ++p)
    if (m[p] < 0 || n[p] < 0 || m[p] > INT32_MAX || n[p] > INT32_MAX) return 0;
  return (size_t)layout_of(count, count_tiles(count, m, n, alpha, table)).total;
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
  gb_batch_tuning def[GB_BATCH_BUCKETS];
  if (!table) {
    gb_sgemv_batch_default_tuning(def);
    table = def;
  }
  for (int b = 0; b < GB_BATCH_BUCKETS; ++b)
    if (!tuning_ok(table[b])) return -9;
  std::vector<Interval> outs, ins;
  for (int64_t p = 0; p < count; ++p) {
    if (m[p] < 0 || m[p] > INT32_MAX) return -2;
    if (n[p] < 0 || n[p] > INT32_MAX) return -3;
    if (lda[p] < (n[p] > 1 ? n[p] : 1)) return -4;
    if (!active(m[p], n[p], alpha[p])) continue;
    if (!A[p]) return -6;
    if (!x[p]) return -7;
    if (!c[p]) return -8;
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(A[p]);
    const uintptr_t x0 = reinterpret_cast<uintptr_t>(x[p]);
    const uintptr_t c0 = reinterpret_cast<uintptr_t>(c[p]);
    const unsigned __int128 ab = ((unsigned __int128)(m[p] - 1) * (uint64_t)lda[p] + (uint64_t)n[p]) * 4u;
    if (ab > (unsigned __int128)(UINTPTR_MAX - a0)) return -4;  // A would run past the address space
    ins.push_back({a0, a0 + (uintptr_t)ab});
    ins.push_back({x0, x0 + (uintptr_t)(n[p] * 4)});
    outs.push_back({c0, c0 + (uintptr_t)(m[p] * 4)});
  }
  auto by_lo = [](const Interval& a, const Interval& b) { return a.lo < b.lo; };
  std::sort(outs.begin(), outs.end(), by_lo);
  for (size_t i = 1; i < outs.size(); ++i)
    if (outs[i].lo < outs[i - 1].hi) return -8;  // two problems write the same c
  std::sort(ins.begin(), ins.end(), by_lo);
  if (meets(outs, ins)) return -8;               // a c overlaps some A or x
  if (!plan || !aligned16(plan)) return -10;

  const int64_t T = count_tiles(count, m, n, alpha, table);
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
    BatchProblem& pb = probs[p];
    pb.A = A[p];
    pb.x = x[p];
    pb.c = c[p];
    pb.lda = lda[p];
    pb.m = (int32_t)m[p];
    pb.n = (int32_t)n[p];
    pb.alpha = alpha[p];
    pb.vec = aligned16(A[p]) && aligned16(x[p]) && lda[p] % 4 == 0;
    if (!active(m[p], n[p], alpha[p])) continue;
    const gb_batch_tuning& tu = table[bucket_of(n[p])];
    const int64_t R = tile_rows(n[p], tu);
    for (int64_t r0 = 0; r0 < m[p]; r0 += R) {
      BatchTile& tl = tiles[t];
      tl.A = A[p] + r0 * lda[p];
      tl.x = x[p];
      tl.c = c[p] + r0;
      tl.lda = lda[p];
      tl.rows = (int32_t)std::min<int64_t>(R, m[p] - r0);
      tl.n = (int32_t)n[p];
      tl.alpha = alpha[p];
      tl.lpr_log2 = (uint8_t)log2_exact(tu.lanes_per_row);
      tl.u_log2 = (uint8_t)log2_exact(tu.packs_per_iter);
      tl.vec = (uint8_t)pb.vec;
      prefix[t] = cost;
      cost += (int64_t)tl.rows * (4 * n[p] + 8) + 4 * n[p] + kTileOverhead;
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
