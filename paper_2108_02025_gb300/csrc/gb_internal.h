// Host-side plumbing shared by the kernel files and the C ABI (api.cu).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "gb_split.h"
#include "gbblas.h"

namespace gb {

constexpr int kThreads = 256;  // every kernel runs 256-thread blocks

template <typename T>
struct GemvArgs {
  int64_t m, n;
  T alpha;
  const T* A;
  int64_t lda;
  const T* x;
  T* c;
};

// Tuning constants shared by the planner (api.cu) and the kernels.
constexpr int kRowLongU = 4;     // packs in flight per thread, long-row kernel (FP32)
constexpr int kRowLongU64 = 8;   // the same for FP64
constexpr int kRowLongD64 = 4;   // of those, packs formed on the FP64 pipe (the rest emulated)
constexpr int kRowLongB64 = 4;   // FP64 long-row kernel: resident blocks per SM budgeted for
constexpr int kRowHeld = 4;      // split long rows: units per block whose arrival waits for the block's end
// FP64 long rows (at least kRowMultiMinRows): R rows per unit share each load
// and cut of x; U packs per row in flight, D of them on the FP64 pipe; B
// resident blocks per SM.
constexpr int kRowMultiR = 2;
constexpr int kRowMultiU = 4;
constexpr int kRowMultiD = 0;
constexpr int kRowMultiB = 4;
constexpr int kRowMultiMinRows = 16;  // fewer FP64 rows take the one-row long kernel
constexpr int kRowShortD64 = 2;  // FP64 short rows: of a lane's 8 packs, those on the FP64 pipe
constexpr int kRowShortB64 = 3;  // FP64 short rows: resident blocks per SM budgeted for
// Short rows: the next row block's packs loaded while the current one is
// summed (FP64, FP32), and the resident blocks per SM budgeted for then.
constexpr bool kRowShortPf64 = false;
constexpr bool kRowShortPf32 = true;
constexpr int kRowShortPfB = 2;
constexpr int64_t kRowShortPPL = 8;  // short rows: packs per lane the lanes per row are sized for (<= 8)
constexpr int kRowScalarRW = 4;  // rows per lane group, misaligned row-major kernel
constexpr int kColTileU = 8;     // columns in flight per thread, column-major tile kernel
constexpr int kColTileD64 = 4;   // FP64: of those, columns formed on the FP64 pipe (the rest emulated)
constexpr int kColTileD64Short = 2;  // the same for tiles of 128 or more rows (n <= kColShortN)
// Column-major GEMVs whose rows fit one tile and whose columns are split:
// CTAs per thread-block cluster (partials summed in distributed shared
// memory, one partial per cluster left for the final sum).
constexpr int kColCluster = 8;
constexpr int kColClusterU32 = 10;  // FP32: columns in flight per thread in that launch
constexpr int64_t kColShortN = 512;  // column-major: n up to this takes tiles of up to 256 row threads
constexpr int64_t kColMinUnits = 1;  // column-major: split until at least this many units per block
constexpr int64_t kRowMinUnits = 2;  // row-major long rows: the same
// BF16 / E4M3 GEMV (index: 0 BF16, 1 E4M3): rows sharing each load of x,
// 16-byte packs per row in flight per thread, and resident blocks per SM
// the registers are budgeted for.
constexpr int kQuantRows[2] = {4, 4};
constexpr int kQuantPacks[2] = {2, 1};
constexpr int kQuantMinBlocks[2] = {2, 3};
constexpr int kQuantE4M3U = 8;  // E4M3 quantiser: 16-byte packs in flight per thread

// How one GEMV is cut into work.  The kernel, the split S and the per-thread
// summation order depend only on (dtype, layout, m, n) and on the pointer
// alignment (which selects the 16-byte or the scalar variant).
struct GemvPlan {
  enum Kind { kRowLong, kRowShort, kRowShift, kRowShortShift, kRowScalar, kCol };
  Kind kind;
  bool vec;         // 16-byte packs (A, x 16-byte aligned and lda a multiple of the pack)
  bool long_chain;  // FP32 only: a thread sums more than 64 products of one row
  bool multi;       // FP64 long rows: the kernel with kRowMultiR rows per unit
  int lpr;          // row-major short / scalar: lanes per row (1..32)
  int txw;          // column-major: lanes along the rows of a warp item (1..32)
  int cluster;      // column-major block tiles: CTAs per cluster summing their partials in
                    // distributed shared memory (0: none); units are then the column chunks
  int64_t kc;       // columns per chunk
  int64_t units;    // work units (kRowLong: m * S; warp kernels: items * S)
  Split split;      // S chunks of the summed index (S = 1: no split) and their workspace
};

template <typename T>
struct DotArgs {
  int64_t n;
  const T* x;
  const T* y;
  T* alpha;
};

struct DotPlan {
  bool vec;
  int64_t chunk;   // elements per block
  int64_t blocks;  // number of blocks (1 = the single-block form, Alg. 3)
  double* part;
  unsigned* ticket;
};

template <typename T>
struct GerArgs {
  int64_t m, n;
  T alpha;
  const T* x;
  const T* y;
  T* C;
  int64_t ldc;
};

struct GerPlan {
  bool vec;
  bool row;        // row-major: lines are rows
  int64_t lines, len;
};

// Blocks to launch for `units` independent work units: `waves` times the
// blocks that fit on the GPU at once (every SM filled to the kernel's
// occupancy), never more blocks than units.  With waves > 1 a block that
// finishes early is replaced by the next one, which evens out the end of
// the launch when blocks stream at different rates.
int grid_size(const void* kernel, int64_t units, size_t smem = 0, int waves = 1);
// Waves of the FP64 kernels (measured on GB300): the row-group kernel and
// the column tile kernel with FP64 products.
constexpr int kRowMultiWaves = 8;
constexpr int kColTileWaves64 = 4;

// Batched level-2 problems (batch.cu): gb_batch_item kinds, and the
// planner behind gb_sgemv_batch_plan / gb_batch_plan with the statuses of
// gb_sgemv_batch_plan (argument numbers of its FP32 form).
constexpr int kBatchGemvF32 = GB_BATCH_GEMV_F32;
constexpr int kBatchGemvBF16 = GB_BATCH_GEMV_BF16;
constexpr int kBatchGerF32 = GB_BATCH_GER_F32;
constexpr int kBatchDotF32 = GB_BATCH_DOT_F32;
using BatchItem = gb_batch_item;
size_t batch_plan_bytes(int64_t count, const BatchItem* items, const gb_batch_tuning* table);
int batch_plan(int64_t count, const BatchItem* items, const gb_batch_tuning* table, void* plan,
               size_t plan_bytes);

// Host-side fault injection (GB_FAULT_INJECT=<site>:<k>): true on the k-th
// call for that site.  Sites: the gb_op codes of gemv, dot, ger, and a step
// of the serving engine.
constexpr int kInjectStep = 3;
constexpr int kInjectSites = 4;
bool fault_injected(int site);

// Allow `kernel` `bytes` of dynamic shared memory on the current device
// (once per kernel and device).  Returns false if the device refuses.
bool allow_smem(const void* kernel, size_t bytes);

template <typename T>
int gemv_row_launch(const GemvArgs<T>& a, const GemvPlan& p, cudaStream_t st);
template <typename T>
int gemv_col_launch(const GemvArgs<T>& a, const GemvPlan& p, cudaStream_t st);
template <typename T>
int dot_launch(const DotArgs<T>& a, const DotPlan& p, cudaStream_t st);
template <typename T>
int ger_launch(const GerArgs<T>& a, const GerPlan& p, cudaStream_t st);

int quantize_bf16_launch(int64_t m, int64_t n, const float* A, int64_t lda, uint16_t* Q,
                         int64_t ldq, cudaStream_t st);
int quantize_e4m3_launch(int64_t m, int64_t n, const float* A, int64_t lda, uint8_t* Q,
                         int64_t ldq, float* scales, cudaStream_t st);
// fmt 0: BF16, 1: E4M3 with per-row scales
int gemv_q_launch(int fmt, int64_t m, int64_t n, float alpha, const void* Q, int64_t ldq,
                  const float* scales, const float* x, float* c, const Split& sp, int64_t kc,
                  int64_t units, cudaStream_t st);

}  // namespace gb
