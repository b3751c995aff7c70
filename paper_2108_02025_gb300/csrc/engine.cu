// Serving engine: continuous batching of GEMV / DOT / GER requests on one
// GPU under an HBM budget (include/gbserve.h).  Not part of the paper, whose
// operations run one call at a time (Sec. 4); a step launches one operand
// kernel (operands drawn by the generator; for requests on the resident
// pools the copies of their initial outputs and their GERs, out of place)
// and one batched level-2 kernel (batch.cu) for all its requests.
//
// One worker thread owns the device side: it admits arrived requests in
// arrival order while the arena and the in-flight cap allow, launches the
// admitted ones as a step on a free stream, and retires steps whose event
// has completed.  Submission and polling only touch mutex-guarded queues.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <set>
#include <thread>
#include <vector>

#include <cuda_bf16.h>

#include "gbblas.h"
#include "gbserve.h"
#include "gb_internal.h"

namespace gb {
namespace {

// ------------------------------------------------------------- generator ---
// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) used as a counter hash.

constexpr uint64_t kG = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kM1 = 0xBF58476D1CE4E5B9ull;
constexpr uint64_t kM2 = 0x94D049BB133111EBull;
constexpr uint64_t kS = 0xD1B54A32D192ED03ull;

__host__ __device__ inline uint64_t sm_mix(uint64_t z) {
  z ^= z >> 30;
  z *= kM1;
  z ^= z >> 27;
  z *= kM2;
  return z ^ (z >> 31);
}

inline uint64_t stream_key(uint64_t seed, uint64_t stream) { return sm_mix(sm_mix(seed + kG) ^ (stream * kS)); }

enum SegKind : int32_t { kFillF32 = 0, kFillBF16 = 1, kCopyF32 = 2, kGerF32 = 3 };

// One piece of a step's operand work.  Fill: count generator values into
// dst.  Copy: dst[k] = src[k].  GER (out of place): dst = src + alpha x y^T
// over count = rows * ld elements, row r = k / ld, column j = k % ld, one
// fma per element with t_j = fl(alpha * y_j); columns n <= j < ld copy src.
struct OperandSeg {  // 64 bytes
  void* dst;
  const float* src;
  const float* x;
  const float* y;
  int64_t count;  // elements written
  uint64_t key;   // fill: generator key; GER: ld (a multiple of 4)
  int32_t kind;
  int32_t n;      // GER: columns
  float alpha;    // GER
  int32_t pad;
};
static_assert(sizeof(OperandSeg) == 64, "operand segment layout");

constexpr int64_t kFillChunk = 16384;  // elements per block (a multiple of 4)

// Elements 2k and 2k+1 of a stream come from one word u = mix(key + (k+1) G):
// bits 63..40 and bits 39..16, each b mapped to b * 2^-23 - 1.  The map is
// done on the bit pattern: 1 + m * 2^-23 (m = the low 23 bits of b) is a
// binary32 in [1, 2), and subtracting 1 (b >= 2^23) or 2 (b < 2^23) is exact.
__device__ __forceinline__ float uniform_of(unsigned b24) {
  const float one_m = __uint_as_float(0x3F800000u | (b24 & 0x7FFFFFu));
  return __fsub_rn(one_m, (b24 & 0x800000u) ? 1.0f : 2.0f);
}

__device__ __forceinline__ void pair_of(uint64_t key, int64_t k, float& v0, float& v1) {
  const uint64_t u = sm_mix(key + (uint64_t)(k + 1) * kG);
  v0 = uniform_of((unsigned)(u >> 40));
  v1 = uniform_of((unsigned)(u >> 16) & 0xFFFFFFu);
}

__device__ __forceinline__ uint16_t bf16_bits(float v) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  return *reinterpret_cast<const uint16_t*>(&h);
}

// Block b works on chunk b - first[s] of segment s, the last s with
// first[s] <= b: four consecutive elements per thread and step, 16-byte
// (FP32) or 8-byte (BF16) accesses.  Fill and GER segments start 16-byte
// aligned (arena pieces 256 bytes, pool operands 32 bytes, GER rows ld a
// multiple of 4 elements apart), so a group of four never straddles a row;
// a copy of the c of a row chunk may start anywhere.
__global__ void __launch_bounds__(kThreads) operand_kernel(const OperandSeg* __restrict__ segs,
                                                           const int64_t* __restrict__ first, int nseg) {
  const int64_t b = blockIdx.x;
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  const OperandSeg sg = segs[lo];
  const int64_t e0 = (b - first[lo]) * kFillChunk;
  const int64_t e1 = e0 + kFillChunk < sg.count ? e0 + kFillChunk : sg.count;
  if (sg.kind == kFillF32 || sg.kind == kFillBF16) {
    for (int64_t e = e0 + 4 * (int64_t)threadIdx.x; e < e1; e += 4 * kThreads) {
      float v[4];
      pair_of(sg.key, e >> 1, v[0], v[1]);
      pair_of(sg.key, (e >> 1) + 1, v[2], v[3]);
      if (sg.kind == kFillF32) {
        float* d = static_cast<float*>(sg.dst) + e;
        if (e + 4 <= e1) {
          *reinterpret_cast<float4*>(d) = make_float4(v[0], v[1], v[2], v[3]);
        } else {
          for (int q = 0; q < 4 && e + q < e1; ++q) d[q] = v[q];
        }
      } else {
        uint16_t* d = static_cast<uint16_t*>(sg.dst) + e;
        if (e + 4 <= e1) {
          const unsigned lo2 = bf16_bits(v[0]) | ((unsigned)bf16_bits(v[1]) << 16);
          const unsigned hi2 = bf16_bits(v[2]) | ((unsigned)bf16_bits(v[3]) << 16);
          *reinterpret_cast<uint2*>(d) = make_uint2(lo2, hi2);
        } else {
          for (int q = 0; q < 4 && e + q < e1; ++q) d[q] = bf16_bits(v[q]);
        }
      }
    }
  } else if (sg.kind == kCopyF32) {
    // a chunk of rows starts at any element: 16-byte accesses only when
    // both ends are 16-byte aligned
    float* d = static_cast<float*>(sg.dst);
    const bool wide = ((reinterpret_cast<uintptr_t>(d) | reinterpret_cast<uintptr_t>(sg.src)) & 15) == 0;
    for (int64_t e = e0 + 4 * (int64_t)threadIdx.x; e < e1; e += 4 * kThreads) {
      if (wide && e + 4 <= e1) {
        *reinterpret_cast<float4*>(d + e) = __ldcs(reinterpret_cast<const float4*>(sg.src + e));
      } else {
        for (int q = 0; q < 4 && e + q < e1; ++q) d[e + q] = sg.src[e + q];
      }
    }
  } else {
    float* d = static_cast<float*>(sg.dst);
    const int64_t ld = (int64_t)sg.key;
    const bool narrow = sg.count <= (int64_t)UINT32_MAX;
    for (int64_t e = e0 + 4 * (int64_t)threadIdx.x; e < e1; e += 4 * kThreads) {
      const int64_t r = narrow ? (int64_t)((uint32_t)e / (uint32_t)ld) : e / ld;
      const int64_t j = e - r * ld;
      const float xr = __ldg(sg.x + r);
      if (e + 4 <= e1 && j + 4 <= sg.n) {
        const float4 y4 = __ldg(reinterpret_cast<const float4*>(sg.y + j));
        float4 c = __ldcs(reinterpret_cast<const float4*>(sg.src + e));
        c.x = __fmaf_rn(xr, __fmul_rn(sg.alpha, y4.x), c.x);
        c.y = __fmaf_rn(xr, __fmul_rn(sg.alpha, y4.y), c.y);
        c.z = __fmaf_rn(xr, __fmul_rn(sg.alpha, y4.z), c.z);
        c.w = __fmaf_rn(xr, __fmul_rn(sg.alpha, y4.w), c.w);
        *reinterpret_cast<float4*>(d + e) = c;
      } else {
        for (int q = 0; q < 4 && e + q < e1; ++q) {
          const float c = sg.src[e + q];
          d[e + q] = j + q < sg.n ? __fmaf_rn(xr, __fmul_rn(sg.alpha, __ldg(sg.y + j + q)), c) : c;
        }
      }
    }
  }
}

// ----------------------------------------------------------------- arena ---

constexpr size_t kAlign = 256;

inline size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// First-fit allocator over [0, cap) with coalescing free ranges.
class Arena {
 public:
  void init(size_t cap) {
    cap_ = cap;
    free_.clear();
    free_[0] = cap;
    used_ = peak_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = round_up(bytes, kAlign);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const size_t rest = it->second - bytes;
      const size_t at = it->first + bytes;
      free_.erase(it);
      if (rest) free_[at] = rest;
      used_ += bytes;
      peak_ = std::max(peak_, used_);
      return true;
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = round_up(bytes, kAlign);
    used_ -= bytes;
    auto next = free_.lower_bound(off);
    size_t start = off, len = bytes;
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        start = prev->first;
        len += prev->second;
        free_.erase(prev);
      }
    }
    if (next != free_.end() && off + bytes == next->first) {
      len += next->second;
      free_.erase(next);
    }
    free_[start] = len;
  }
  size_t used() const { return used_; }
  size_t peak() const { return peak_; }

 private:
  std::map<size_t, size_t> free_;
  size_t cap_ = 0, used_ = 0, peak_ = 0;
};

// -------------------------------------------------------------- requests ---

struct Piece {
  size_t off, bytes;  // inside the request's range
};

// Layout of a request's operands: leading dimensions and 256-byte pieces.
struct Footprint {
  int64_t ld = 0;
  Piece p[3] = {};  // GEMV: A|Q, x, c; DOT: x, y, alpha; GER: C, x, y
                    // (from the pool: the output alone, c, alpha or C)
  int pieces = 0;
  size_t total = 0;
  int64_t extent[3] = {};  // elements of operand streams 1, 2, 3
};

inline bool pooled(const gb_request& r) { return (r.flags & GB_REQ_POOL) != 0; }

inline bool request_ok(const gb_request& r) {
  if ((r.flags & ~GB_REQ_POOL) != 0) return false;
  if (r.n < 1 || r.n > INT32_MAX) return false;
  switch (r.op) {
    case GB_REQ_GEMV:
      return (r.form == GB_FORM_F32 || r.form == GB_FORM_BF16) && r.m >= 1 && r.m <= INT32_MAX;
    case GB_REQ_GER:
      return r.form == GB_FORM_F32 && r.m >= 1 && r.m <= INT32_MAX;
    case GB_REQ_DOT:
      return r.form == GB_FORM_F32;
    default:
      return false;
  }
}

Footprint footprint(const gb_request& r) {
  Footprint f;
  auto add = [&](size_t bytes) {
    f.p[f.pieces++] = Piece{f.total, bytes};
    f.total += round_up(bytes > 0 ? bytes : 1, kAlign);
  };
  const size_t m = (size_t)r.m, n = (size_t)r.n;
  const bool pool = pooled(r);
  if (r.op == GB_REQ_GEMV) {
    f.ld = (int64_t)round_up(n, r.form == GB_FORM_BF16 ? 8 : 4);
    f.extent[0] = (int64_t)(m * (size_t)f.ld);
    f.extent[1] = (int64_t)n;
    f.extent[2] = (int64_t)m;
    if (!pool) {
      add(m * (size_t)f.ld * (r.form == GB_FORM_BF16 ? 2 : 4));
      add(n * 4);
    }
    add(m * 4);
  } else if (r.op == GB_REQ_DOT) {
    f.ld = (int64_t)round_up(n, 4);
    f.extent[0] = f.extent[1] = (int64_t)n;
    f.extent[2] = 1;
    if (!pool) {
      add((size_t)f.ld * 4);  // x (leading dimension rounded up like a GEMV row)
      add(n * 4);
    }
    add(4);
  } else {
    f.ld = (int64_t)round_up(n, 4);
    f.extent[0] = (int64_t)(m * (size_t)f.ld);
    f.extent[1] = (int64_t)m;
    f.extent[2] = (int64_t)n;
    add(m * (size_t)f.ld * 4);
    if (!pool) {
      add(m * 4);
      add(n * 4);
    }
  }
  return f;
}

// Start (elements) of operand stream s in a pool of P elements:
// 8 * (mix(key(seed, s)) mod (floor((P - L) / 8) + 1)), L <= P.
inline int64_t pool_offset(uint64_t seed, uint64_t s, int64_t extent, int64_t P) {
  const uint64_t slots = (uint64_t)((P - extent) / 8) + 1;
  return (int64_t)(8 * (sm_mix(stream_key(seed, s)) % slots));
}

struct Req {
  gb_request r;
  Footprint f;
  int64_t pool_off[3] = {};  // GB_REQ_POOL: element offsets of operand streams 1, 2, 3
  size_t off = 0;
  unsigned char* base = nullptr;  // device address of the range (host-only: nullptr)
  int64_t admit_ns = 0, launch_ns = 0, done_ns = 0, step = -1;
  int status = GB_OK;
  // Launch in row chunks (GEMV and GER on the pool, larger than the chunk
  // size): rows launched so far, parts whose step has not retired, and the
  // (slot, step) of every part launched.
  int64_t rows = 1, rows_launched = 0, row_bytes = 0;
  bool chunked = false;
  int parts_out = 0;
  std::vector<std::pair<int, int64_t>> part_steps;
  unsigned char* ptr(int i) const { return base + f.p[i].off; }
};

// Rows [row0, row0 + rows) of a request, launched in one step; `last` is
// the part that completes the request's rows (its step copies the result).
struct Part {
  Req* q;
  int64_t row0, rows;
  bool last;
};

constexpr int64_t kSpinNs = 200000;  // the worker polls instead of sleeping this close to an arrival

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// ------------------------------------------------------------------ slots ---

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  unsigned char* host = nullptr;  // pinned staging of the step's descriptors
  unsigned char* dev = nullptr;
  size_t cap = 0;
  bool busy = false;
  int64_t index = -1;
  int64_t sim_done_ns = 0;  // host-only mode
  bool failed = false;
  int fail_status = GB_OK;
  std::vector<Part> parts;
};

}  // namespace
}  // namespace gb

using namespace gb;

struct gb_engine {
  gb_engine_config cfg{};
  gb_batch_tuning table[GB_BATCH_BUCKETS];
  bool host_only = false;
  unsigned char* arena_base = nullptr;
  float* pool_f32 = nullptr;      // resident operands (GB_REQ_POOL)
  uint16_t* pool_bf16 = nullptr;
  size_t pool_bytes = 0;
  Arena arena;
  std::vector<Slot> slots;

  std::mutex mu;  // guards pending, done, counters, stop
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> pending;  // sorted by arrival
  std::deque<gb_completion> done;
  bool stop = false;
  int64_t submitted = 0, completed = 0, failed = 0;

  // worker-only state
  std::deque<Req*> admitted;
  int64_t inflight = 0;
  // written by the worker, read by gb_engine_stats_get
  std::atomic<int64_t> inflight_peak{0}, steps{0}, steps_inflight_peak{0};
  std::atomic<int64_t> admitted_count{0};
  std::atomic<size_t> bytes_in_use{0}, bytes_peak{0};
  std::thread worker;

  void run();
  bool retire();
  bool admit();
  bool launch();
  int launch_step(Slot& s, const std::vector<Part>& parts);
  int ensure_capacity(Slot& s, size_t bytes);
  void finish(Slot& s, int64_t t, int status);
};

// Retire every step whose work has completed.
bool gb_engine::retire() {
  bool any = false;
  for (Slot& s : slots) {
    if (!s.busy) continue;
    int status = GB_OK;
    if (s.failed) {
      status = s.fail_status;
    } else if (host_only) {
      if (now_ns() < s.sim_done_ns) continue;
    } else {
      const cudaError_t q = cudaEventQuery(s.done);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) {
        cudaGetLastError();
        status = GB_ERR_CUDA;
      }
    }
    finish(s, now_ns(), status);
    any = true;
  }
  return any;
}

// A step has retired: its parts are done.  A request completes when all its
// rows have been launched and no part of it is still on the GPU.
void gb_engine::finish(Slot& s, int64_t t, int status) {
  std::vector<gb_completion> out;
  for (const Part& pt : s.parts) {
    Req* q = pt.q;
    if (status != GB_OK && q->status == GB_OK) q->status = status;
    if (--q->parts_out > 0 || q->rows_launched < q->rows) continue;
    q->done_ns = t;
    arena.release(q->off, q->f.total);
    gb_completion c{};
    c.id = q->r.id;
    c.status = q->status;
    c.op = q->r.op;
    c.arrival_ns = q->r.arrival_ns;
    c.admitted_ns = q->admit_ns;
    c.launched_ns = q->launch_ns;
    c.done_ns = t;
    c.step = q->step;
    c.bytes = (int64_t)q->f.total;
    out.push_back(c);
    delete q;
    --inflight;
  }
  s.parts.clear();
  s.busy = false;
  s.failed = false;
  bytes_in_use = arena.used();
  {
    std::lock_guard<std::mutex> lk(mu);
    for (const gb_completion& c : out) {
      done.push_back(c);
      ++completed;
      if (c.status != GB_OK) ++failed;
    }
  }
  cv_done.notify_all();
}

// Admit arrived requests in arrival order while memory and the cap allow.
bool gb_engine::admit() {
  bool any = false;
  const int64_t t = now_ns();
  std::lock_guard<std::mutex> lk(mu);
  while (!pending.empty()) {
    Req* q = pending.front();
    if ((q->r.arrival_ns > t && !stop) || inflight >= cfg.max_inflight) break;
    size_t off = 0;
    if (!arena.alloc(q->f.total, &off)) break;  // head of line waits for memory
    q->off = off;
    q->base = host_only ? nullptr : arena_base + off;
    q->admit_ns = t;
    admitted.push_back(q);
    pending.pop_front();
    ++inflight;
    ++admitted_count;
    if (inflight > inflight_peak.load()) inflight_peak = inflight;
    any = true;
  }
  bytes_in_use = arena.used();
  bytes_peak = arena.peak();
  return any;
}

int gb_engine::ensure_capacity(Slot& s, size_t bytes) {
  if (bytes <= s.cap) return GB_OK;
  const size_t cap = round_up(std::max(bytes, 2 * s.cap), 1 << 16);
  if (s.host) cudaFreeHost(s.host);
  if (s.dev) cudaFree(s.dev);
  s.host = nullptr;
  s.dev = nullptr;
  s.cap = 0;
  if (cudaHostAlloc(&s.host, cap, cudaHostAllocDefault) != cudaSuccess) return GB_ERR_CUDA;
  if (cudaMalloc(&s.dev, cap) != cudaSuccess) return GB_ERR_CUDA;
  s.cap = cap;
  return GB_OK;
}

// Enqueue one step: descriptors, one operand kernel (operands drawn by the
// generator; for pool requests the copies of the initial outputs and the
// GERs), one batched launch for the GEMVs and DOTs (and the GERs of drawn
// requests), result copies, event.
int gb_engine::launch_step(Slot& s, const std::vector<Part>& parts) {
  std::vector<OperandSeg> segs;
  auto fill = [&](void* dst, int64_t count, uint64_t key, int32_t kind) {
    OperandSeg g{};
    g.dst = dst;
    g.count = count;
    g.key = key;
    g.kind = kind;
    segs.push_back(g);
  };
  for (const Part& pt : parts) {
    const Req* q = pt.q;
    const gb_request& r = q->r;
    const uint64_t seed = r.seed;
    if (pooled(r)) {  // rows [row0, row0 + rows) of the output
      const float* P = pool_f32;
      OperandSeg g{};
      if (r.op == GB_REQ_GER) {
        g.dst = reinterpret_cast<float*>(q->ptr(0)) + pt.row0 * q->f.ld;
        g.src = P + q->pool_off[0] + pt.row0 * q->f.ld;
        g.x = P + q->pool_off[1] + pt.row0;
        g.y = P + q->pool_off[2];
        g.count = pt.rows * q->f.ld;
        g.key = (uint64_t)q->f.ld;
        g.kind = kGerF32;
        g.n = (int32_t)r.n;
        g.alpha = r.alpha;
      } else {
        g.dst = reinterpret_cast<float*>(q->ptr(0)) + pt.row0;
        g.src = P + q->pool_off[2] + pt.row0;
        g.count = pt.rows;
        g.kind = kCopyF32;
      }
      segs.push_back(g);
    } else if (r.op == GB_REQ_GEMV) {  // drawn requests are never split
      fill(q->ptr(0), r.m * q->f.ld, stream_key(seed, 1), r.form == GB_FORM_BF16 ? kFillBF16 : kFillF32);
      fill(q->ptr(1), r.n, stream_key(seed, 2), kFillF32);
      fill(q->ptr(2), r.m, stream_key(seed, 3), kFillF32);
    } else if (r.op == GB_REQ_DOT) {
      fill(q->ptr(0), r.n, stream_key(seed, 1), kFillF32);
      fill(q->ptr(1), r.n, stream_key(seed, 2), kFillF32);
      fill(q->ptr(2), 1, stream_key(seed, 3), kFillF32);
    } else {
      fill(q->ptr(0), r.m * q->f.ld, stream_key(seed, 1), kFillF32);
      fill(q->ptr(1), r.m, stream_key(seed, 2), kFillF32);
      fill(q->ptr(2), r.n, stream_key(seed, 3), kFillF32);
    }
  }
  std::vector<int64_t> first(segs.size() + 1, 0);
  for (size_t i = 0; i < segs.size(); ++i)
    first[i + 1] = first[i] + (segs[i].count + kFillChunk - 1) / kFillChunk;

  // every GEMV (FP32 or BF16 A) and DOT (FP32 Dot2 per thread, the final
  // sum in FP64) in one batched launch, with the GERs of drawn requests
  std::vector<BatchItem> items;
  items.reserve(parts.size());
  for (const Part& pt : parts) {
    const Req* q = pt.q;
    const gb_request& r = q->r;
    const bool pool = pooled(r);
    if (pool && r.op == GB_REQ_GER) continue;  // done by the operand kernel
    BatchItem it{};
    it.n = r.n;
    it.lda = q->f.ld;
    if (pool) {
      const float* P = pool_f32;
      it.kind = r.op == GB_REQ_DOT ? kBatchDotF32
                : r.form == GB_FORM_BF16 ? kBatchGemvBF16 : kBatchGemvF32;
      it.m = r.op == GB_REQ_GEMV ? pt.rows : 1;
      it.alpha = r.op == GB_REQ_GEMV ? r.alpha : 1.0f;
      // GEMV and DOT kinds only read A; rows [row0, row0 + rows)
      const int64_t a0 = q->pool_off[0] + pt.row0 * q->f.ld;
      it.A = it.kind == kBatchGemvBF16 ? static_cast<void*>(pool_bf16 + a0) : static_cast<void*>(pool_f32 + a0);
      it.x = P + q->pool_off[1];
      it.c = reinterpret_cast<float*>(q->ptr(0)) + pt.row0;
    } else if (r.op == GB_REQ_GEMV) {
      it.kind = r.form == GB_FORM_BF16 ? kBatchGemvBF16 : kBatchGemvF32;
      it.m = r.m;
      it.alpha = r.alpha;
      it.A = q->ptr(0);
      it.x = reinterpret_cast<const float*>(q->ptr(1));
      it.c = reinterpret_cast<float*>(q->ptr(2));
    } else if (r.op == GB_REQ_DOT) {
      it.kind = kBatchDotF32;
      it.m = 1;
      it.alpha = 1.0f;
      it.A = q->ptr(0);
      it.x = reinterpret_cast<const float*>(q->ptr(1));
      it.c = reinterpret_cast<float*>(q->ptr(2));
    } else {
      it.kind = kBatchGerF32;
      it.m = r.m;
      it.alpha = r.alpha;
      it.A = q->ptr(0);                                    // C
      it.x = reinterpret_cast<const float*>(q->ptr(2));  // y
      it.c = reinterpret_cast<float*>(q->ptr(1));        // x
    }
    items.push_back(it);
  }
  const int64_t nb = (int64_t)items.size();
  const size_t plan_bytes = batch_plan_bytes(nb, items.data(), table);
  if (plan_bytes == 0) return GB_ERR_UNSUPPORTED;

  // staging layout: segs | first | plan
  const size_t o_first = round_up(segs.size() * sizeof(OperandSeg), 16);
  const size_t o_plan = round_up(o_first + first.size() * sizeof(int64_t), 256);
  const size_t total = o_plan + plan_bytes;
  int st = ensure_capacity(s, total);
  if (st != GB_OK) return st;
  std::memcpy(s.host, segs.data(), segs.size() * sizeof(OperandSeg));
  std::memcpy(s.host + o_first, first.data(), first.size() * sizeof(int64_t));
  st = batch_plan(nb, items.data(), table, s.host + o_plan, plan_bytes);
  if (st != GB_OK) return GB_ERR_UNSUPPORTED;
  cudaStream_t sm = s.stream;
  if (cudaMemcpyAsync(s.dev, s.host, total, cudaMemcpyHostToDevice, sm) != cudaSuccess) return GB_ERR_CUDA;
  if (!segs.empty()) {
    const int64_t blocks = first.back();
    operand_kernel<<<(unsigned)blocks, kThreads, 0, sm>>>(reinterpret_cast<const OperandSeg*>(s.dev),
                                                          reinterpret_cast<const int64_t*>(s.dev + o_first),
                                                          (int)segs.size());
    if (cudaPeekAtLastError() != cudaSuccess) return GB_ERR_CUDA;
  }
  if (nb > 0 && gb_sgemv_batch(s.host + o_plan, s.dev + o_plan, sm) != GB_OK) return GB_ERR_CUDA;
  for (const Part& pt : parts) {
    const Req* q = pt.q;
    const gb_request& r = q->r;
    if (!r.out || !pt.last) continue;
    // the result is whole once the request's earlier parts, on other
    // streams, are done too
    for (const auto& ps : q->part_steps) {
      const Slot& o = slots[(size_t)ps.first];
      if (&o != &s && o.busy && o.index == ps.second && !o.failed)
        if (cudaStreamWaitEvent(sm, o.done, 0) != cudaSuccess) return GB_ERR_CUDA;
    }
    cudaError_t e;
    const unsigned char* res = pooled(r) || r.op == GB_REQ_GER ? q->ptr(0) : q->ptr(2);
    if (r.op == GB_REQ_GER)
      e = cudaMemcpy2DAsync(r.out, (size_t)r.n * 4, res, (size_t)q->f.ld * 4, (size_t)r.n * 4, (size_t)r.m,
                            cudaMemcpyDeviceToHost, sm);
    else
      e = cudaMemcpyAsync(r.out, res, r.op == GB_REQ_DOT ? 4 : (size_t)r.m * 4, cudaMemcpyDeviceToHost, sm);
    if (e != cudaSuccess) return GB_ERR_CUDA;
  }
  if (cudaEventRecord(s.done, sm) != cudaSuccess) return GB_ERR_CUDA;
  return GB_OK;
}

// Launch admitted requests as a step on a free slot.  Whole requests first,
// in admission order (at most max_step_requests); then, with a chunk size
// set, row chunks of the chunked requests in admission order until the step
// holds chunk_bytes of their work, so a large request never holds the GPU
// for longer than a chunk while smaller ones wait behind it.
bool gb_engine::launch() {
  if (admitted.empty()) return false;
  Slot* s = nullptr;
  int busy = 0, slot = -1;
  for (size_t i = 0; i < slots.size(); ++i) {
    if (slots[i].busy) ++busy;
    else if (!s) {
      s = &slots[i];
      slot = (int)i;
    }
  }
  if (!s) return false;
  std::vector<Part> parts;
  size_t whole = 0;
  for (auto it = admitted.begin(); it != admitted.end() && whole < (size_t)cfg.max_step_requests;) {
    Req* q = *it;
    if (q->chunked) {
      ++it;
      continue;
    }
    parts.push_back(Part{q, 0, q->rows, true});
    q->rows_launched = q->rows;
    ++whole;
    it = admitted.erase(it);
  }
  int64_t room = (int64_t)cfg.chunk_bytes;
  for (auto it = admitted.begin(); it != admitted.end() && room > 0;) {
    Req* q = *it;
    if (!q->chunked) {
      ++it;
      continue;
    }
    const int64_t left = q->rows - q->rows_launched;
    int64_t take = room / q->row_bytes;
    if (take < 1) take = 1;
    if (take > left) take = left;
    parts.push_back(Part{q, q->rows_launched, take, q->rows_launched + take == q->rows});
    q->rows_launched += take;
    room -= take * q->row_bytes;
    if (q->rows_launched == q->rows) it = admitted.erase(it);
    else ++it;
  }
  if (parts.empty()) return false;
  s->parts = parts;
  s->index = steps++;
  s->busy = true;
  if (busy + 1 > steps_inflight_peak.load()) steps_inflight_peak = busy + 1;
  const int64_t t = now_ns();
  size_t bytes = 0;
  int64_t after = 0;  // host-only: the step ends after the earlier parts of its requests
  for (const Part& pt : s->parts) {
    Req* q = pt.q;
    if (q->parts_out == 0 && q->step < 0) q->launch_ns = t;
    q->step = s->index;
    ++q->parts_out;
    bytes += q->chunked ? (size_t)(pt.rows * q->row_bytes) : q->f.total;
    if (pt.last)
      for (const auto& ps : q->part_steps)
        if (slots[(size_t)ps.first].busy && slots[(size_t)ps.first].index == ps.second)
          after = std::max(after, slots[(size_t)ps.first].sim_done_ns);
    q->part_steps.emplace_back(slot, s->index);
  }
  if (fault_injected(kInjectStep)) {
    s->failed = true;
    s->fail_status = GB_ERR_INJECTED;
    return true;
  }
  if (host_only) {
    s->sim_done_ns = std::max(after, t + (int64_t)((double)bytes / cfg.sim_bytes_per_ns));
    return true;
  }
  const int st = launch_step(*s, s->parts);
  if (st != GB_OK) {
    // nothing more is enqueued on this stream; let what was enqueued finish
    cudaStreamSynchronize(s->stream);
    cudaGetLastError();
    s->failed = true;
    s->fail_status = st == GB_ERR_CUDA ? GB_ERR_CUDA : st;
  }
  return true;
}

void gb_engine::run() {
  for (;;) {
    bool progress = retire();
    progress |= admit();
    progress |= launch();
    bool busy = false;
    for (const Slot& s : slots) busy |= s.busy;
    std::unique_lock<std::mutex> lk(mu);
    if (stop && pending.empty() && admitted.empty() && !busy) break;
    if (progress) continue;
    // Steps on the GPU, or an arrival due within kSpinNs: poll again at
    // once (a timed sleep overshoots by tens of microseconds, which would
    // add to every request's latency); otherwise sleep until shortly before
    // the next arrival, or until a submission.
    const int64_t wait = pending.empty() ? INT64_MAX : pending.front()->r.arrival_ns - now_ns();
    if (busy || wait <= kSpinNs) {
      lk.unlock();
      std::this_thread::yield();
      continue;
    }
    if (!pending.empty()) {
      cv_work.wait_for(lk, std::chrono::nanoseconds(std::min<int64_t>(wait - kSpinNs, 1000000)));
    } else if (!stop) {
      cv_work.wait_for(lk, std::chrono::milliseconds(1));
    }
  }
}

namespace {

// Allocate the operand pools and draw them (FP32: stream 1 of the pool seed;
// BF16: stream 2, rounded) on the first slot's stream; returns when done.
int fill_pool(gb_engine* e) {
  const int64_t P = e->cfg.pool_elems;
  if (cudaMalloc(&e->pool_f32, (size_t)P * 4) != cudaSuccess) return GB_ERR_CUDA;
  if (cudaMalloc(&e->pool_bf16, (size_t)P * 2) != cudaSuccess) return GB_ERR_CUDA;
  e->pool_bytes = (size_t)P * 6;
  OperandSeg segs[2] = {};
  segs[0].dst = e->pool_f32;
  segs[0].count = P;
  segs[0].key = stream_key(e->cfg.pool_seed, 1);
  segs[0].kind = kFillF32;
  segs[1].dst = e->pool_bf16;
  segs[1].count = P;
  segs[1].key = stream_key(e->cfg.pool_seed, 2);
  segs[1].kind = kFillBF16;
  const int64_t per = (P + kFillChunk - 1) / kFillChunk;
  const int64_t first[3] = {0, per, 2 * per};
  unsigned char* d = nullptr;
  if (cudaMalloc(&d, 256) != cudaSuccess) return GB_ERR_CUDA;
  cudaStream_t sm = e->slots[0].stream;
  int st = GB_OK;
  if (cudaMemcpyAsync(d, segs, sizeof(segs), cudaMemcpyHostToDevice, sm) != cudaSuccess ||
      cudaMemcpyAsync(d + 128, first, sizeof(first), cudaMemcpyHostToDevice, sm) != cudaSuccess) {
    st = GB_ERR_CUDA;
  } else {
    operand_kernel<<<(unsigned)(2 * per), kThreads, 0, sm>>>(reinterpret_cast<const OperandSeg*>(d),
                                                            reinterpret_cast<const int64_t*>(d + 128), 2);
    if (cudaPeekAtLastError() != cudaSuccess) st = GB_ERR_CUDA;
  }
  if (cudaStreamSynchronize(sm) != cudaSuccess) st = GB_ERR_CUDA;
  cudaFree(d);
  return st;
}

}  // namespace

extern "C" {

int64_t gb_engine_now_ns(void) { return now_ns(); }

size_t gb_engine_request_bytes(const gb_request* r) {
  if (!r || !request_ok(*r)) return 0;
  return footprint(*r).total;
}

int gb_engine_create(const gb_engine_config* cfg, gb_engine** out) {
  if (!cfg) return -1;
  if (!out) return -2;
  *out = nullptr;
  if (cfg->budget_bytes < ((size_t)1 << 20) || cfg->streams < 1 || cfg->streams > 16 ||
      cfg->max_inflight < 1 || cfg->max_step_requests < 1 || (cfg->flags & ~GB_ENGINE_HOST_ONLY) != 0 ||
      cfg->pool_elems < 0 || cfg->pool_elems % 8 != 0 || cfg->pool_elems > ((int64_t)1 << 40))
    return -1;
  const bool host_only = (cfg->flags & GB_ENGINE_HOST_ONLY) != 0;
  if (host_only && !(cfg->sim_bytes_per_ns > 0.0)) return -1;
  gb_engine* e = new gb_engine();
  e->cfg = *cfg;
  e->host_only = host_only;
  if (cfg->table) std::memcpy(e->table, cfg->table, sizeof(e->table));
  else gb_sgemv_batch_default_tuning(e->table);
  e->cfg.table = e->table;
  {  // validate the table with a one-problem plan size
    const int64_t one = 1;
    const float a = 1.f;
    if (gb_sgemv_batch_plan_bytes(1, &one, &one, &a, e->table) == 0) {
      delete e;
      return -1;
    }
  }
  e->arena.init(cfg->budget_bytes);
  e->slots.resize((size_t)cfg->streams);
  if (!host_only) {
    bool ok = cudaMalloc(&e->arena_base, cfg->budget_bytes) == cudaSuccess;
    for (Slot& s : e->slots) {
      if (!ok) break;
      ok = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) == cudaSuccess;
    }
    if (ok && cfg->pool_elems > 0) ok = fill_pool(e) == GB_OK;
    if (!ok) {
      cudaGetLastError();
      for (Slot& s : e->slots) {
        if (s.done) cudaEventDestroy(s.done);
        if (s.stream) cudaStreamDestroy(s.stream);
      }
      if (e->arena_base) cudaFree(e->arena_base);
      if (e->pool_f32) cudaFree(e->pool_f32);
      if (e->pool_bf16) cudaFree(e->pool_bf16);
      delete e;
      return GB_ERR_CUDA;
    }
  }
  int dev = 0;
  if (!host_only) cudaGetDevice(&dev);
  try {
    e->worker = std::thread([e, dev, host_only] {
      if (!host_only) cudaSetDevice(dev);
      e->run();
    });
  } catch (...) {
    for (Slot& s : e->slots) {
      if (s.done) cudaEventDestroy(s.done);
      if (s.stream) cudaStreamDestroy(s.stream);
    }
    if (e->arena_base) cudaFree(e->arena_base);
    if (e->pool_f32) cudaFree(e->pool_f32);
    if (e->pool_bf16) cudaFree(e->pool_bf16);
    delete e;
    return GB_ERR_CUDA;
  }
  *out = e;
  return GB_OK;
}

int gb_engine_submit(gb_engine* e, const gb_request* r) {
  if (!e) return -1;
  if (!r || !request_ok(*r)) return -2;
  if (r->out && !e->host_only) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, r->out) != cudaSuccess || at.type != cudaMemoryTypeHost) {
      cudaGetLastError();
      return -2;
    }
  }
  Req* q = new Req();
  q->r = *r;
  q->f = footprint(*r);
  if (pooled(*r)) {
    const int64_t P = e->cfg.pool_elems;
    for (int k = 0; k < 3; ++k) {
      if (q->f.extent[k] > P) {
        delete q;
        return -2;
      }
      q->pool_off[k] = pool_offset(r->seed, (uint64_t)(k + 1), q->f.extent[k], P);
    }
  }
  if (q->f.total > e->cfg.budget_bytes) {
    delete q;
    return GB_ERR_BUDGET;
  }
  q->rows = r->op == GB_REQ_DOT ? 1 : r->m;
  if (pooled(*r) && r->op != GB_REQ_DOT && e->cfg.chunk_bytes > 0) {
    // bytes a row moves: the A row and c (GEMV), the C0 and C rows (GER)
    const int64_t eb = r->op == GB_REQ_GEMV && r->form == GB_FORM_BF16 ? 2 : 4;
    q->row_bytes = r->op == GB_REQ_GEMV ? q->f.ld * eb + 8 : q->f.ld * 8;
    q->chunked = q->row_bytes * q->rows > (int64_t)e->cfg.chunk_bytes;
  }
  if (q->r.arrival_ns == 0) q->r.arrival_ns = now_ns();
  {
    std::lock_guard<std::mutex> lk(e->mu);
    auto pos = std::upper_bound(e->pending.begin(), e->pending.end(), q->r.arrival_ns,
                                [](int64_t t, const Req* x) { return t < x->r.arrival_ns; });
    e->pending.insert(pos, q);
    ++e->submitted;
  }
  e->cv_work.notify_one();
  return GB_OK;
}

int gb_engine_poll(gb_engine* e, gb_completion* out, int max) {
  if (!e || max < 0 || (max > 0 && !out)) return -1;
  std::lock_guard<std::mutex> lk(e->mu);
  int k = 0;
  while (k < max && !e->done.empty()) {
    out[k++] = e->done.front();
    e->done.pop_front();
  }
  return k;
}

int gb_engine_drain(gb_engine* e, int64_t timeout_ms) {
  if (!e || timeout_ms < 0) return -1;
  std::unique_lock<std::mutex> lk(e->mu);
  const bool ok = e->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                      [e] { return e->completed == e->submitted; });
  return ok ? GB_OK : GB_ERR_TIMEOUT;
}

int gb_engine_stats_get(gb_engine* e, gb_engine_stats* out) {
  if (!e || !out) return -1;
  std::lock_guard<std::mutex> lk(e->mu);
  out->submitted = e->submitted;
  out->admitted = e->admitted_count.load();
  out->completed = e->completed;
  out->failed = e->failed;
  out->steps = e->steps.load();
  out->inflight_peak = e->inflight_peak.load();
  out->steps_inflight_peak = e->steps_inflight_peak.load();
  out->bytes_in_use = e->bytes_in_use.load();
  out->bytes_peak = e->bytes_peak.load();
  out->budget_bytes = e->cfg.budget_bytes;
  out->pool_bytes = e->pool_bytes;
  return 0;
}

void gb_engine_destroy(gb_engine* e) {
  if (!e) return;
  gb_engine_drain(e, 60000);
  {
    std::lock_guard<std::mutex> lk(e->mu);
    e->stop = true;
  }
  e->cv_work.notify_all();
  if (e->worker.joinable()) e->worker.join();
  std::set<Req*> owned(e->pending.begin(), e->pending.end());
  owned.insert(e->admitted.begin(), e->admitted.end());
  for (Slot& s : e->slots) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    for (const Part& pt : s.parts) owned.insert(pt.q);
    if (s.done) cudaEventDestroy(s.done);
    if (s.stream) cudaStreamDestroy(s.stream);
    if (s.host) cudaFreeHost(s.host);
    if (s.dev) cudaFree(s.dev);
  }
  for (Req* q : owned) delete q;
  if (e->arena_base) cudaFree(e->arena_base);
  if (e->pool_f32) cudaFree(e->pool_f32);
  if (e->pool_bf16) cudaFree(e->pool_bf16);
  delete e;
}

}  // extern "C"
