// C ABI of the library (declared in include/gbblas.h): argument checks,
// work plans, workspace layout and kernel dispatch.  Host code only; nothing
// here allocates, frees or synchronises.
#include <atomic>
#include <cuda.h>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "gbblas.h"
#include "gb_internal.h"

namespace gb {
namespace {

// Warps resident at once in the pipelined GEMV kernels on GB300: 152 SMs x
// 2 blocks x 8 warps (shared memory allows two blocks per SM).
constexpr int64_t kWaveWarps = 2432;
constexpr int kMaxSplits = 4096;
// DOT is one block (Alg. 3) while one vector holds at most this many bytes,
// else blocks of the index range (Alg. 4); the crossover measured on GB300
// (dot_cutoff.py).  A compile-time constant so that studies can rebuild it.
#ifndef GB_DOT_SMALL_BYTES
#define GB_DOT_SMALL_BYTES 65536
#endif
constexpr int64_t kDotSmallBytes = GB_DOT_SMALL_BYTES;
constexpr int64_t kDotBlocks = 608;     // large DOT: at most this many blocks (Alg. 4)
constexpr int kDotPack = 4;             // packs per thread per step in the DOT kernel

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t pow2_at_least(int64_t v, int64_t cap) {
  int64_t p = 1;
  while (p < v && p < cap) p <<= 1;
  return p;
}
inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// [lo, hi) byte ranges overlap?
inline bool overlap(const void* a, unsigned __int128 abytes, const void* b, unsigned __int128 bbytes) {
  if (abytes == 0 || bbytes == 0) return false;
  const unsigned __int128 a0 = reinterpret_cast<uintptr_t>(a), b0 = reinterpret_cast<uintptr_t>(b);
  return a0 < b0 + bbytes && b0 < a0 + abytes;
}

// Bytes spanned by an m x n matrix with leading dimension ld.
inline unsigned __int128 matrix_bytes(int layout, int64_t m, int64_t n, int64_t ld, size_t e) {
  if (m == 0 || n == 0) return 0;
  const unsigned __int128 lines = layout == GB_ROW_MAJOR ? m : n;
  const unsigned __int128 len = layout == GB_ROW_MAJOR ? n : m;
  return ((lines - 1) * (unsigned __int128)ld + len) * e;
}

// ---------------------------------------------------------------- plans ---

struct SplitShape {
  int S, G, NG;
  int64_t kc, items;
};

inline size_t ticket_bytes(const SplitShape& s) {
  return ((size_t)s.items * (s.NG + 1) * sizeof(unsigned) + 255) / 256 * 256;
}

inline size_t split_bytes(const SplitShape& s, int64_t m) {
  if (s.S <= 1) return 0;
  return ticket_bytes(s) + (size_t)s.S * m * sizeof(double) +
         (s.NG > 1 ? (size_t)s.NG * m * sizeof(double) : 0);
}

inline Split split_view(const SplitShape& s, int64_t m, void* ws) {
  Split sp{s.S, s.G, s.NG, m, nullptr, nullptr, nullptr};
  if (s.S <= 1) return sp;
  char* base = static_cast<char*>(ws);
  sp.tickets = reinterpret_cast<unsigned*>(base);
  sp.part = reinterpret_cast<double*>(base + ticket_bytes(s));
  sp.part2 = s.NG > 1 ? sp.part + (size_t)s.S * m : nullptr;
  return sp;
}

inline int64_t isqrt_ceil(int64_t v) {
  int64_t r = 1;
  while (r * r < v) ++r;
  return r;
}

// Number of chunks of the summed index (length n, element size e) for
// `items` row items.  The items * S warp work items are spread over the
// kWaveWarps warps that fit on the GPU at once: S is the smallest split count
// whose last wave is at least 95% full (else the fullest), with chunks of at
// least `min_kc` indices (multiples of `quantum`) and the partial sums'
// traffic (16 bytes per row per chunk) under 1% of the matrix's.  Depends
// only on the shape.
inline SplitShape choose_split(int64_t items, int64_t n, int64_t min_kc, int64_t quantum, size_t e) {
  SplitShape s{1, 1, 1, n > 0 ? n : 1, items};
  int64_t smax = kMaxSplits;
  if (smax > n / min_kc) smax = n / min_kc;
  if (smax > n * (int64_t)e / 1600) smax = n * (int64_t)e / 1600;
  auto fill = [&](int64_t S) {
    const int64_t u = items * S;
    return (double)u / (double)(cdiv(u, kWaveWarps) * kWaveWarps);
  };
  int64_t best = 1;
  double best_fill = fill(1);
  if (best_fill < 0.95) {
    for (int64_t S = 2; S <= smax; ++S) {
      const double f = fill(S);
      if (f > best_fill + 1e-9) { best = S; best_fill = f; }
      if (f >= 0.95) break;
    }
  }
  if (best < 2) return s;
  const int64_t kc = cdiv(cdiv(n, best), quantum) * quantum;
  const int64_t S = cdiv(n, kc);
  if (S < 2) return s;
  s.S = (int)S;
  s.G = S <= 32 ? (int)S : (int)isqrt_ceil(S);  // one level up to 32 partials
  s.NG = (int)cdiv(S, s.G);
  s.kc = kc;
  return s;
}

inline int64_t pow2_floor(int64_t v) {
  int64_t p = 1;
  while (p * 2 <= v) p <<= 1;
  return p;
}

// Blocks resident at once in the block-streaming GEMV kernels on GB300: 152
// SMs x 4 blocks of 256 threads.
constexpr int64_t kWaveBlocks = 608;

// Split count for the block-streaming kernels, whose blocks take equal
// consecutive ranges of `items * S` units: the smallest S giving at least
// 4 units per block with the busiest block at most 5% above the average,
// else the most even S (units below one per block are penalised).  Chunks
// hold at least `min_kc` indices (multiples of `quantum`); the partials'
// traffic (16 bytes per row per chunk) stays under 1% of the matrix's.
// `wave` is the number of blocks resident at once.  Depends only on the
// shape.
inline SplitShape block_split(int64_t items, int64_t n, int64_t min_kc, int64_t quantum, size_t e,
                              int64_t wave = kWaveBlocks, int64_t min_units = 4) {
  SplitShape s{1, 1, 1, n > 0 ? n : 1, items};
  int64_t smax = kMaxSplits;
  if (smax > n / min_kc) smax = n / min_kc;
  if (smax > n * (int64_t)e / 1600) smax = n * (int64_t)e / 1600;
  auto even = [&](int64_t S) {
    const double u = (double)(items * S) / wave;  // units per block, average
    const double busiest = (double)cdiv(items * S, wave);
    return (u / busiest) * (u < 1.0 ? u : 1.0);
  };
  if (items >= min_units * wave || smax < 2) return s;
  int64_t best = 1;
  double best_even = even(1);
  for (int64_t S = 2; S <= smax; ++S) {
    const double ev = even(S);
    if (items * S >= min_units * wave && ev >= 0.95) { best = S; break; }
    if (ev > best_even + 1e-9) { best = S; best_even = ev; }
  }
  if (best < 2) return s;
  const int64_t kc = cdiv(cdiv(n, best), quantum) * quantum;
  const int64_t S = cdiv(n, kc);
  if (S < 2) return s;
  s.S = (int)S;
  s.G = S <= 32 ? (int)S : (int)isqrt_ceil(S);
  s.NG = (int)cdiv(S, s.G);
  s.kc = kc;
  return s;
}

struct RowShape {
  GemvPlan::Kind kind;
  int lpr;
  bool long_chain;
  bool multi;  // FP64 long rows in groups of kRowMultiR
  SplitShape sp;
};

// al: 2 = A rows and x 16-byte aligned (16-byte packs), 1 = x 16-byte
// aligned and A element-aligned but its rows not on 16 bytes (long rows are
// read realigned), 0 = anything else (scalar loads).
inline RowShape row_shape(size_t e, int al, int64_t m, int64_t n) {
  const bool vec = al == 2;
  if (al == 1 && cdiv(n, 16 / (int64_t)e) > 256) {  // long rows, realigned packs
    RowShape r{};
    const int64_t V = 16 / (int64_t)e;
    const int64_t quantum = 256 * V;
    r.kind = GemvPlan::kRowShift;
    SplitShape s = block_split(m, n, quantum * kRowLongU, quantum, e, kWaveBlocks, kRowMinUnits);
    s.G = s.S;  // one counter per row, as the long-row kernel
    s.NG = 1;
    r.sp = s;
    r.long_chain = e == 4 && cdiv(s.kc, 256 * V) * V > 64;
    return r;
  }
  if (al == 1) {  // short rows, realigned packs (lane groups as for aligned short rows)
    RowShape r{};
    const int64_t packs = cdiv(n, 16 / (int64_t)e);
    r.kind = GemvPlan::kRowShortShift;
    r.lpr = (int)pow2_at_least(cdiv(packs, kRowShortPPL), 32);
    r.sp = SplitShape{1, 1, 1, n, cdiv(m, 256 / r.lpr)};
    return r;
  }
  const int64_t V = vec ? 16 / (int64_t)e : 1;
  RowShape r{};
  const int64_t packs = cdiv(n, V);
  if (vec && packs <= 256) {  // short rows: lane groups of up to 8 packs each, no split
    r.kind = GemvPlan::kRowShort;
    r.lpr = (int)pow2_at_least(cdiv(packs, kRowShortPPL), 32);
    r.sp = SplitShape{1, 1, 1, n, cdiv(m, 256 / r.lpr)};
    return r;
  }
  if (vec && e == 8 && m >= kRowMultiMinRows) {  // FP64 long rows: (row group, chunk) units
    r.kind = GemvPlan::kRowLong;
    r.multi = true;
    const int64_t quantum = 256 * V;
    SplitShape s = block_split(cdiv(m, kRowMultiR), n, quantum * kRowMultiU, quantum, e, 152 * kRowMultiB,
                               kRowMinUnits);
    s.G = s.S;  // one counter per row group, the group's S partials summed in one level
    s.NG = 1;
    r.sp = s;
    return r;
  }
  if (vec) {  // long rows: blocks stream (row, chunk) units; one counter per row
    r.kind = GemvPlan::kRowLong;
    const int64_t quantum = 256 * V;
    SplitShape s = block_split(m, n, quantum * (e == 8 ? kRowLongU64 : kRowLongU), quantum, e, kWaveBlocks,
                               kRowMinUnits);
    s.G = s.S;   // the long-row kernel sums a row's S partials in one level
    s.NG = 1;
    r.sp = s;
    r.long_chain = e == 4 && cdiv(s.kc, 256 * V) * V > 64;
    return r;
  }
  r.kind = GemvPlan::kRowScalar;  // misaligned operands
  int64_t lpr = pow2_floor(packs / 8 > 0 ? packs / 8 : 1);
  r.lpr = (int)(lpr > 32 ? 32 : lpr);
  const int64_t rows = (32 / r.lpr) * kRowScalarRW;
  r.sp = choose_split(cdiv(m, rows), n, r.lpr * 8, 1, e);
  return r;
}

struct ColShape {
  int txw;
  bool long_chain;
  int cluster = 0;     // CTAs per cluster (kColCluster) or 0
  int64_t chunks = 0;  // cluster > 0: column chunks (= blocks); sp then describes the cluster partials
  SplitShape sp;
};

constexpr int kColU = 8;  // columns unrolled, misaligned column-major kernel (gemv_col.cu)

inline ColShape col_shape(size_t e, bool vec, int64_t m, int64_t n) {
  const int64_t V = vec ? 16 / (int64_t)e : 1;
  ColShape c;
  if (vec) {  // block tiles of tx*V rows; tx threads along the rows, 256/tx along the columns
    // short columns (n small): up to all 256 threads along the rows, no
    // cross-lane sum (FP64: up to 128, so that a tile is smaller and the
    // last wave of tiles shorter, unless n <= 32, where two column lanes
    // would leave each thread too few columns for its fixed cost per tile:
    // 2097152x32 102.8 -> 94.1 us with 256, 1048576x64 89.3 -> 91.6 us);
    // otherwise at most 64
    const int64_t txs = e == 8 ? (n <= 32 ? 256 : 128) : 256;
    const int64_t tx = pow2_at_least(cdiv(m, V), n <= kColShortN ? txs : 64);
    const int64_t ty = 256 / tx;
    c.txw = (int)tx;
    c.sp = block_split(cdiv(m, tx * V), n, ty * kColTileU, 1, e, kWaveBlocks, kColMinUnits);
    if (c.sp.items == 1 && c.sp.S > 1 && tx * V <= 256) {
      // one row tile, columns split: chunks in clusters of kColCluster CTAs,
      // one partial per cluster (a single level of the final sum)
      const int64_t chunks = cdiv(c.sp.S, kColCluster) * kColCluster;
      const int64_t kc = cdiv(n, chunks);
      c.cluster = kColCluster;
      c.chunks = chunks;
      const int64_t parts = chunks / kColCluster;
      c.sp.S = (int)parts;
      c.sp.G = (int)parts;
      c.sp.NG = 1;
      c.sp.kc = kc;
    }
    c.long_chain = e == 4 && cdiv(c.sp.kc, ty) > 64;
    return c;
  }
  // misaligned operands: warp items; at most 32 row lanes, no more than the rows need
  const int64_t txw = pow2_at_least(cdiv(m, V), 32);
  const int64_t tyw = 32 / txw;
  c.txw = (int)txw;
  c.sp = choose_split(cdiv(m, txw * V), n, tyw * kColU * 2, 1, e);
  c.long_chain = e == 4 && cdiv(c.sp.kc, tyw) > 64;
  return c;
}

inline void dot_shape(size_t e, bool vec, int64_t n, int64_t* chunk, int64_t* blocks) {
  if (n <= kDotSmallBytes / (int64_t)e) {
    *chunk = n;
    *blocks = 1;
    return;
  }
  const int64_t V = vec ? 16 / (int64_t)e : 1;
  const int64_t q = 256 * V * kDotPack;
  int64_t G = cdiv(n, q);
  if (G > kDotBlocks) G = kDotBlocks;
  *chunk = cdiv(cdiv(n, G), q) * q;
  *blocks = cdiv(n, *chunk);
}

inline size_t dot_bytes(int64_t blocks) {
  return blocks <= 1 ? 0 : 256 + (size_t)blocks * sizeof(double);
}

// The workspace size does not depend on pointer alignment: both variants
// are sized and the larger is reported.
size_t gemv_ws(size_t e, int layout, int64_t m, int64_t n) {
  size_t b = 0;
  for (int al = 0; al < 3; ++al) {
    const SplitShape s = layout == GB_ROW_MAJOR ? row_shape(e, al, m, n).sp : col_shape(e, al == 2, m, n).sp;
    const size_t w = split_bytes(s, m);
    if (w > b) b = w;
  }
  return b;
}

size_t dot_ws(size_t e, int64_t n) {
  size_t b = 0;
  for (int vec = 0; vec < 2; ++vec) {
    int64_t chunk, blocks;
    dot_shape(e, vec, n, &chunk, &blocks);
    const size_t w = dot_bytes(blocks);
    if (w > b) b = w;
  }
  return b;
}

// Reduced-precision GEMV (row-major): items are groups of kQuantRows rows,
// one counter per group; `per` elements per 16-byte pack.
inline SplitShape qgemv_shape(int fmt, int64_t m, int64_t n) {
  const int64_t per = fmt == 0 ? 8 : 16;
  const int64_t quantum = 256 * per;
  SplitShape s = block_split(cdiv(m, kQuantRows[fmt]), n, quantum * kQuantPacks[fmt], quantum,
                             fmt == 0 ? 2 : 1, 152 * kQuantMinBlocks[fmt]);
  s.G = s.S;
  s.NG = 1;
  return s;
}

// ------------------------------------------------------- fault injection ---

struct Inject {
  int op = -1;
  long long nth = 0;
  std::atomic<long long> count[kInjectSites] = {0, 0, 0, 0};
};

Inject& inject() {
  static Inject inj;
  static std::once_flag once;
  std::call_once(once, [] {
    const char* v = std::getenv("GB_FAULT_INJECT");
    if (!v) return;
    const char* colon = std::strchr(v, ':');
    if (!colon) return;
    const size_t len = (size_t)(colon - v);
    if (len == 4 && std::strncmp(v, "gemv", 4) == 0) inj.op = GB_OP_GEMV;
    else if (len == 3 && std::strncmp(v, "dot", 3) == 0) inj.op = GB_OP_DOT;
    else if (len == 3 && std::strncmp(v, "ger", 3) == 0) inj.op = GB_OP_GER;
    else if (len == 4 && std::strncmp(v, "step", 4) == 0) inj.op = kInjectStep;
    inj.nth = std::atoll(colon + 1);
  });
  return inj;
}

inline bool injected(int op) {
  Inject& inj = inject();
  const long long k = inj.count[op].fetch_add(1) + 1;
  return inj.op == op && k == inj.nth;
}

inline int cuda_status() {
  return cudaPeekAtLastError() == cudaSuccess ? GB_OK : GB_ERR_CUDA;
}

// ------------------------------------------------------------- dispatch ---

// No work between the checks and the launch (gb_dgemv, gb_sgemv).
struct NoPrelaunch {
  int operator()() const { return GB_OK; }
};

// `pre` runs after every argument check and the fault-injection check,
// immediately before the launch; a status other than GB_OK from it is
// returned with nothing launched.
template <typename T, typename Pre = NoPrelaunch>
int gemv(int layout, int64_t m, int64_t n, T alpha, const T* A, int64_t lda, const T* x, T* c,
         void* ws, size_t ws_bytes, gb_stream stream, Pre pre = Pre{}) {
  if (layout != GB_ROW_MAJOR && layout != GB_COL_MAJOR) return -1;
  if (m < 0) return -2;
  if (n < 0) return -3;
  const int64_t min_ld = layout == GB_ROW_MAJOR ? (n > 1 ? n : 1) : (m > 1 ? m : 1);
  if (lda < min_ld) return -6;
  if (m == 0 || n == 0 || alpha == T(0)) return GB_OK;
  if (!A) return -5;
  if (!x) return -7;
  if (!c) return -8;
  const size_t e = sizeof(T);
  const unsigned __int128 cb = (unsigned __int128)m * e;
  if (overlap(c, cb, A, matrix_bytes(layout, m, n, lda, e)) || overlap(c, cb, x, (unsigned __int128)n * e))
    return -8;
  const size_t need = gemv_ws(e, layout, m, n);
  if (need > 0 && (!ws || !aligned16(ws))) return -9;
  if (ws_bytes < need) return GB_ERR_WORKSPACE;
  if (injected(GB_OP_GEMV)) return GB_ERR_INJECTED;
  if (const int st = pre(); st != GB_OK) return st;

  const int64_t V = 16 / (int64_t)e;
  const bool vec = aligned16(A) && aligned16(x) && lda % V == 0;
  const int al = vec ? 2 : (aligned16(x) && reinterpret_cast<uintptr_t>(A) % e == 0) ? 1 : 0;
  GemvArgs<T> a{m, n, alpha, A, lda, x, c};
  GemvPlan p{};
  p.vec = vec;
  SplitShape s;
  if (layout == GB_ROW_MAJOR) {
    const RowShape r = row_shape(e, al, m, n);
    p.kind = r.kind;
    p.lpr = r.lpr;
    p.long_chain = r.long_chain;
    s = r.sp;
    p.multi = r.multi;
  } else {
    const ColShape cs = col_shape(e, vec, m, n);
    p.kind = GemvPlan::kCol;
    p.txw = cs.txw;
    p.long_chain = cs.long_chain;
    p.cluster = cs.cluster;
    s = cs.sp;
  }
  p.kc = s.kc;
  p.units = s.items * s.S;
  if (p.cluster > 0) p.units = s.S * (int64_t)p.cluster;  // one column chunk per CTA
  p.split = split_view(s, m, ws);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (layout == GB_ROW_MAJOR) gemv_row_launch<T>(a, p, st);
  else gemv_col_launch<T>(a, p, st);
  return cuda_status();
}

template <typename T>
int dot(int64_t n, const T* x, const T* y, T* alpha, void* ws, size_t ws_bytes, gb_stream stream) {
  if (n < 0) return -1;
  if (n == 0) return GB_OK;
  if (!x) return -2;
  if (!y) return -3;
  if (!alpha) return -4;
  const size_t e = sizeof(T);
  if (overlap(alpha, e, x, (unsigned __int128)n * e) || overlap(alpha, e, y, (unsigned __int128)n * e))
    return -4;
  const size_t need = dot_ws(e, n);
  if (need > 0 && (!ws || !aligned16(ws))) return -5;
  if (ws_bytes < need) return GB_ERR_WORKSPACE;
  if (injected(GB_OP_DOT)) return GB_ERR_INJECTED;

  DotArgs<T> a{n, x, y, alpha};
  DotPlan p{};
  p.vec = aligned16(x) && aligned16(y);
  dot_shape(e, p.vec, n, &p.chunk, &p.blocks);
  if (p.blocks > 1) {
    p.ticket = static_cast<unsigned*>(ws);
    p.part = reinterpret_cast<double*>(static_cast<char*>(ws) + 256);
  }
  dot_launch<T>(a, p, static_cast<cudaStream_t>(stream));
  return cuda_status();
}

template <typename T>
int ger(int layout, int64_t m, int64_t n, T alpha, const T* x, const T* y, T* C, int64_t ldc,
        gb_stream stream) {
  if (layout != GB_ROW_MAJOR && layout != GB_COL_MAJOR) return -1;
  if (m < 0) return -2;
  if (n < 0) return -3;
  const int64_t min_ld = layout == GB_ROW_MAJOR ? (n > 1 ? n : 1) : (m > 1 ? m : 1);
  if (ldc < min_ld) return -8;
  if (m == 0 || n == 0 || alpha == T(0)) return GB_OK;
  if (!x) return -5;
  if (!y) return -6;
  if (!C) return -7;
  const size_t e = sizeof(T);
  const unsigned __int128 cb = matrix_bytes(layout, m, n, ldc, e);
  if (overlap(C, cb, x, (unsigned __int128)m * e) || overlap(C, cb, y, (unsigned __int128)n * e)) return -7;
  if (injected(GB_OP_GER)) return GB_ERR_INJECTED;

  const int64_t V = 16 / (int64_t)e;
  GerArgs<T> a{m, n, alpha, x, y, C, ldc};
  GerPlan p{};
  p.row = layout == GB_ROW_MAJOR;
  p.lines = p.row ? m : n;
  p.len = p.row ? n : m;
  p.vec = aligned16(C) && ldc % V == 0 && aligned16(p.row ? (const void*)y : (const void*)x);
  ger_launch<T>(a, p, static_cast<cudaStream_t>(stream));
  return cuda_status();
}

// Shared checks of the reduced-precision GEMV entry points.
int qgemv(int fmt, int64_t m, int64_t n, float alpha, const void* Q, int64_t ldq,
          const float* scales, const float* x, float* c, void* ws, size_t ws_bytes,
          gb_stream stream) {
  const int64_t bytes = fmt == 0 ? 2 : 1;
  const int k = fmt == 0 ? 0 : 1;  // E4M3 has the extra scales argument
  if (m < 0) return -1;
  if (n < 0) return -2;
  if (ldq < (n > 1 ? n : 1) || (ldq * bytes) % 16 != 0) return -5;
  if (m == 0 || n == 0 || alpha == 0.f) return GB_OK;
  if (!Q || !aligned16(Q)) return -4;
  if (fmt == 1 && !scales) return -6;
  if (!x || !aligned16(x)) return -(6 + k);
  if (!c) return -(7 + k);
  const unsigned __int128 cb = (unsigned __int128)m * 4;
  if (overlap(c, cb, Q, matrix_bytes(GB_ROW_MAJOR, m, n, ldq, (size_t)bytes)) ||
      overlap(c, cb, x, (unsigned __int128)n * 4) || (fmt == 1 && overlap(c, cb, scales, cb)))
    return -(7 + k);
  const SplitShape s = qgemv_shape(fmt, m, n);
  const size_t need = split_bytes(s, m);
  if (need > 0 && (!ws || !aligned16(ws))) return -(8 + k);
  if (ws_bytes < need) return GB_ERR_WORKSPACE;
  if (injected(GB_OP_GEMV)) return GB_ERR_INJECTED;
  gemv_q_launch(fmt, m, n, alpha, Q, ldq, scales, x, c, split_view(s, m, ws), s.kc, s.items * s.S,
                static_cast<cudaStream_t>(stream));
  return cuda_status();
}

}  // namespace

bool fault_injected(int site) { return injected(site); }

// Occupancy of each kernel is queried once per (kernel, device).
int grid_size(const void* kernel, int64_t units, size_t smem, int waves) {
  struct Entry {
    const void* k;
    int dev;
    int blocks;
  };
  static Entry cache[256];
  static int used = 0;
  static std::mutex mu;
  int dev = 0;
  cudaGetDevice(&dev);
  int blocks = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    for (int i = 0; i < used; ++i)
      if (cache[i].k == kernel && cache[i].dev == dev) blocks = cache[i].blocks;
    if (blocks == 0) {
      int sms = 0, per_sm = 0;
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, smem);
      blocks = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
      if (used < 256) cache[used++] = Entry{kernel, dev, blocks};
    }
  }
  const int64_t want = (int64_t)blocks * (waves > 1 ? waves : 1);
  return (int)(units < want ? (units > 0 ? units : 1) : want);
}

bool allow_smem(const void* kernel, size_t bytes) {
  struct Entry {
    const void* k;
    int dev;
  };
  static Entry done[256];
  static int used = 0;
  static std::mutex mu;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  for (int i = 0; i < used; ++i)
    if (done[i].k == kernel && done[i].dev == dev) return true;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
    return false;
  if (used < 256) done[used++] = Entry{kernel, dev};
  return true;
}

}  // namespace gb

// ------------------------------------------------------------------ C ABI ---

extern "C" {

int gb_version(void) { return 100; }

const char* gb_status_string(int status) {
  switch (status) {
    case GB_OK: return "GB_OK: success";
    case GB_ERR_WORKSPACE: return "GB_ERR_WORKSPACE: workspace smaller than gb_workspace_bytes()";
    case GB_ERR_UNSUPPORTED: return "GB_ERR_UNSUPPORTED: unsupported argument combination";
    case GB_ERR_CUDA: return "GB_ERR_CUDA: kernel launch failed";
    case GB_ERR_INJECTED: return "GB_ERR_INJECTED: fault injected through GB_FAULT_INJECT";
    default: break;
  }
  if (status < 0 && status > -100) return "invalid argument (status -k: argument k)";
  return "unknown status";
}

size_t gb_workspace_bytes(int op, int dtype, int layout, int64_t m, int64_t n) {
  if (op != GB_OP_GEMV_BF16 && op != GB_OP_GEMV_E4M3 && dtype != GB_F32 && dtype != GB_F64) return 0;
  const size_t e = dtype == GB_F32 ? 4 : 8;
  if (op == GB_OP_DOT) return n > 0 ? gb::dot_ws(e, n) : 0;
  if (op == GB_OP_GEMV_BF16 || op == GB_OP_GEMV_E4M3) {
    if (layout != GB_ROW_MAJOR || m <= 0 || n <= 0) return 0;
    return gb::split_bytes(gb::qgemv_shape(op == GB_OP_GEMV_BF16 ? 0 : 1, m, n), m);
  }
  if (op == GB_OP_GEMV) {
    if (layout != GB_ROW_MAJOR && layout != GB_COL_MAJOR) return 0;
    if (m <= 0 || n <= 0) return 0;
    return gb::gemv_ws(e, layout, m, n);
  }
  return 0;
}

int gb_workspace_init(void* ws, size_t ws_bytes, gb_stream stream) {
  if (ws_bytes == 0) return GB_OK;
  if (!ws) return -1;
  return cudaMemsetAsync(ws, 0, ws_bytes, static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? GB_OK
             : GB_ERR_CUDA;
}

int gb_dgemv(int layout, int64_t m, int64_t n, double alpha, const double* A, int64_t lda,
             const double* x, double* c, void* ws, size_t ws_bytes, gb_stream stream) {
  return gb::gemv<double>(layout, m, n, alpha, A, lda, x, c, ws, ws_bytes, stream);
}

int gb_sgemv(int layout, int64_t m, int64_t n, float alpha, const float* A, int64_t lda,
             const float* x, float* c, void* ws, size_t ws_bytes, gb_stream stream) {
  return gb::gemv<float>(layout, m, n, alpha, A, lda, x, c, ws, ws_bytes, stream);
}

int gb_ddot(int64_t n, const double* x, const double* y, double* alpha, void* ws, size_t ws_bytes,
            gb_stream stream) {
  return gb::dot<double>(n, x, y, alpha, ws, ws_bytes, stream);
}

int gb_sdot(int64_t n, const float* x, const float* y, float* alpha, void* ws, size_t ws_bytes,
            gb_stream stream) {
  return gb::dot<float>(n, x, y, alpha, ws, ws_bytes, stream);
}

int gb_dger(int layout, int64_t m, int64_t n, double alpha, const double* x, const double* y,
            double* C, int64_t ldc, gb_stream stream) {
  return gb::ger<double>(layout, m, n, alpha, x, y, C, ldc, stream);
}

int gb_sger(int layout, int64_t m, int64_t n, float alpha, const float* x, const float* y,
            float* C, int64_t ldc, gb_stream stream) {
  return gb::ger<float>(layout, m, n, alpha, x, y, C, ldc, stream);
}

}  // extern "C"

// ------------------------------------------------ reduced precision of A ---

extern "C" {

int gb_quantize_bf16(int64_t m, int64_t n, const float* A, int64_t lda, uint16_t* Q, int64_t ldq,
                     gb_stream stream) {
  if (m < 0) return -1;
  if (n < 0) return -2;
  if (lda < (n > 1 ? n : 1)) return -4;
  if (ldq < (n > 1 ? n : 1)) return -6;
  if (m == 0 || n == 0) return GB_OK;
  if (!A) return -3;
  if (!Q) return -5;
  if (gb::overlap(Q, gb::matrix_bytes(GB_ROW_MAJOR, m, n, ldq, 2), A, gb::matrix_bytes(GB_ROW_MAJOR, m, n, lda, 4)))
    return -5;
  gb::quantize_bf16_launch(m, n, A, lda, Q, ldq, static_cast<cudaStream_t>(stream));
  return gb::cuda_status();
}

int gb_quantize_e4m3(int64_t m, int64_t n, const float* A, int64_t lda, uint8_t* Q, int64_t ldq,
                     float* scales, gb_stream stream) {
  if (m < 0) return -1;
  if (n < 0) return -2;
  if (lda < (n > 1 ? n : 1)) return -4;
  if (ldq < (n > 1 ? n : 1)) return -6;
  if (m == 0 || n == 0) return GB_OK;
  if (!A) return -3;
  if (!Q) return -5;
  if (!scales) return -7;
  const unsigned __int128 ab = gb::matrix_bytes(GB_ROW_MAJOR, m, n, lda, 4);
  if (gb::overlap(Q, gb::matrix_bytes(GB_ROW_MAJOR, m, n, ldq, 1), A, ab)) return -5;
  if (gb::overlap(scales, (unsigned __int128)m * 4, A, ab) ||
      gb::overlap(scales, (unsigned __int128)m * 4, Q, gb::matrix_bytes(GB_ROW_MAJOR, m, n, ldq, 1)))
    return -7;
  gb::quantize_e4m3_launch(m, n, A, lda, Q, ldq, scales, static_cast<cudaStream_t>(stream));
  return gb::cuda_status();
}

int gb_gemv_bf16(int64_t m, int64_t n, float alpha, const uint16_t* Q, int64_t ldq,
                 const float* x, float* c, void* ws, size_t ws_bytes, gb_stream stream) {
  return gb::qgemv(0, m, n, alpha, Q, ldq, nullptr, x, c, ws, ws_bytes, stream);
}

int gb_gemv_e4m3(int64_t m, int64_t n, float alpha, const uint8_t* Q, int64_t ldq,
                 const float* scales, const float* x, float* c, void* ws, size_t ws_bytes,
                 gb_stream stream) {
  return gb::qgemv(1, m, n, alpha, Q, ldq, scales, x, c, ws, ws_bytes, stream);
}

}  // extern "C"

// ------------------------------------------------- GEMV without allocation ---
//
// gb_dgemv_noalloc: the FP64 GEMV of gb_dgemv for callers that cannot call
// cudaMalloc or take memory from an allocator (a runtime that owns the whole
// device heap, or code that must not allocate once set up, for example).
// Its split sums use a scratch array compiled into this library instead of a
// caller-supplied workspace.  Like every entry point here it calls the CUDA
// runtime, so it must not be called from a host callback or stream callback
// (cudaLaunchHostFunc), where CUDA calls are not allowed.

namespace gb {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(256) << 10;  // 256 KiB on every GPU that loads us
constexpr int kNoAllocMaxDevices = 64;

// Lives on each device for the lifetime of the process.  In host code this
// name is only a stand-in: its device address comes from
// cudaGetSymbolAddress (noalloc_scratch below).
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Identity of the calling thread's current context (0 when it cannot be
// told), through the driver entry points the runtime hands out, so that a
// context rebuilt after cudaDeviceReset is seen as a new one.
unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
  });
  if (!get_current || !get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the scratch array in the current context, looked up
// with cudaGetSymbolAddress the first time a context of a device calls, and
// again whenever the device's context has changed since (cudaDeviceReset
// rebuilds it, and the array with it); nullptr on failure.
void* noalloc_scratch() {
  static std::mutex mu;
  static void* addr[kNoAllocMaxDevices] = {};
  static unsigned long long ctx_of[kNoAllocMaxDevices] = {};
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  const unsigned long long ctx = current_context_id();
  if (addr[dev] != nullptr && ctx != 0 && ctx == ctx_of[dev]) return addr[dev];
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return nullptr;
  addr[dev] = p;
  ctx_of[dev] = current_context_id();  // the lookup made the context current if none was
  return p;
}

// Bytes at the start of the workspace that hold arrival counters (they must
// be zero when a call starts), for either pointer-alignment variant.
size_t noalloc_ticket_bytes(int layout, int64_t m, int64_t n) {
  size_t b = 0;
  for (int al = 0; al < 3; ++al) {
    const SplitShape s = layout == GB_ROW_MAJOR ? row_shape(8, al, m, n).sp : col_shape(8, al == 2, m, n).sp;
    if (s.S <= 1) continue;
    const size_t t = ticket_bytes(s);
    if (t > b) b = t;
  }
  return b;
}

}  // namespace
}  // namespace gb

extern "C" int gb_dgemv_noalloc(int layout, int64_t m, int64_t n, double alpha, const double* A,
                                int64_t lda, const double* x, double* c, gb_stream stream) {
  using namespace gb;
  const bool shape_ok = (layout == GB_ROW_MAJOR || layout == GB_COL_MAJOR) && m >= 0 && n >= 0;
  const size_t need = shape_ok && m > 0 && n > 0 ? gemv_ws(sizeof(double), layout, m, n) : 0;
  if (need == 0)  // no split sums: gb_dgemv itself, which needs no workspace here
    return gemv<double>(layout, m, n, alpha, A, lda, x, c, nullptr, 0, stream);
  if (need > kNoAllocScratchBytes) {
    // the built-in scratch is too small: gb_dgemv's checks without a
    // workspace give an invalid argument's own status first, else -9 (the
    // missing workspace), reported as GB_ERR_WORKSPACE; nothing is launched
    const int st = gemv<double>(layout, m, n, alpha, A, lda, x, c, nullptr, 0, stream);
    return st == -9 ? GB_ERR_WORKSPACE : st;
  }
  void* ws = noalloc_scratch();
  if (ws == nullptr) return GB_ERR_CUDA;
  // Once every check has passed (so that a refused or injected call enqueues
  // nothing): zero the counters.  The kernels return them to zero as they
  // finish, so this only matters after a call that did not run to the end or
  // overlapped another one; the array otherwise keeps the last call's data.
  const size_t tb = noalloc_ticket_bytes(layout, m, n);
  return gemv<double>(layout, m, n, alpha, A, lda, x, c, ws, need, stream, [&] {
    if (tb > 0 && cudaMemsetAsync(ws, 0, tb, static_cast<cudaStream_t>(stream)) != cudaSuccess)
      return GB_ERR_CUDA;
    return GB_OK;
  });
}
