// Reduced-precision storage of A for GEMV: BF16, and FP8 E4M3 with one FP32
// scale per row.  Not in the paper (its GEMV is FP64/FP32); fewer bytes of A
// per product is the lever on an HBM-bound GEMV.
//
// * quantisers: BF16 = binary32 rounded to its top 16 bits (nearest, ties
//   to even); E4M3 (OCP FP8: bias 7, 3 mantissa bits, largest finite 448)
//   with s_i = fl32(amax_i / 448) and q_ij = E4M3_rne_satfinite(fl32(A_ij /
//   s_i)); all-zero rows get s_i = 0 and codes 0.
// * GEMV: c_i <- c_i + alpha * s_i * sum_j q_ij x_j (s_i = 1 for BF16), x
//   and c FP32.  Row-major only, streamed like the FP32 long-row kernel (a
//   block per (row group, chunk) unit, interleaved units: block b takes b, b + G, ...); products
//   are FP32 fmas in chains of at most 32, folded into a compensated FP32 sum
//   (TwoSum), then a fixed-order block sum.
#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "gb_common.cuh"
#include "gb_internal.h"

namespace gb {
namespace {

// ------------------------------------------------------------- decoders ---

// BF16 bits -> FP32 (exact).
__device__ __forceinline__ float bf16_bits_to_float(unsigned b) { return __uint_as_float(b << 16); }

// E4M3 bits -> FP32 (exact).  The 7 magnitude bits, moved to the top of a
// binary32 exponent/mantissa field, are the E4M3 value times 2^-120 for
// normals and for subnormals alike (an FP32 subnormal in the second case),
// so one multiplication by 2^120 finishes the job.  The NaN codes 0x7F and
// 0xFF, which the quantiser never writes, are not decoded as NaN.
__device__ __forceinline__ float e4m3_bits_to_float(unsigned b) {
  const float v = __fmul_rn(__uint_as_float((b & 0x7Fu) << 20), 0x1p120f);
  return __uint_as_float(__float_as_uint(v) | ((b & 0x80u) << 24));
}

template <int FMT>  // 0: BF16 (8 per 16-byte pack), 1: E4M3 (16 per pack)
struct Fmt {
  static constexpr int PER = FMT == 0 ? 8 : 16;  // elements per 16-byte pack
  static constexpr int BYTES = FMT == 0 ? 2 : 1;
};

// ------------------------------------------------------------ quantisers ---

// BF16 codes of a row-major FP32 matrix.  A unit is a chunk of kQChunk
// columns of one row; block b takes the units b, b + G, ...  With A and Q
// rows on 16 bytes each thread converts two packs of 8 elements (two 16-byte
// loads, one 16-byte store each); other rows, and the columns past the last
// whole pack, go element by element.  Rounding: __float2bfloat16_rn.
constexpr int64_t kQChunk = (int64_t)kThreads * 16;

__device__ __forceinline__ unsigned bf16_pair(float lo, float hi) {
  const __nv_bfloat16 a = __float2bfloat16_rn(lo), b = __float2bfloat16_rn(hi);
  return (unsigned)*reinterpret_cast<const uint16_t*>(&a) | ((unsigned)*reinterpret_cast<const uint16_t*>(&b) << 16);
}

__global__ void __launch_bounds__(kThreads)
    quantize_bf16_kernel(int64_t m, int64_t n, const float* __restrict__ A, int64_t lda,
                         uint16_t* __restrict__ Q, int64_t ldq, int64_t chunks, bool vec) {
  const int64_t units = m * chunks;
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int64_t i = u / chunks;
    const int64_t k0 = (u - i * chunks) * kQChunk;
    const int64_t k1 = k0 + kQChunk < n ? k0 + kQChunk : n;
    const float* Ar = A + i * lda;
    uint16_t* Qr = Q + i * ldq;
    int64_t kv = k0;  // columns from here on go element by element
    if (vec) {
      const int64_t whole = k0 + (k1 - k0) / 8 * 8;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t j = k0 + ((int64_t)h * kThreads + threadIdx.x) * 8;
        if (j < whole) {
          const float4 a0 = __ldcs(reinterpret_cast<const float4*>(Ar + j));
          const float4 a1 = __ldcs(reinterpret_cast<const float4*>(Ar + j + 4));
          const uint4 q = make_uint4(bf16_pair(a0.x, a0.y), bf16_pair(a0.z, a0.w), bf16_pair(a1.x, a1.y),
                                     bf16_pair(a1.z, a1.w));
          __stcs(reinterpret_cast<uint4*>(Qr + j), q);
        }
      }
      kv = whole;
    }
    for (int64_t j = kv + threadIdx.x; j < k1; j += kThreads) {
      const __nv_bfloat16 b = __float2bfloat16_rn(__ldcs(Ar + j));
      Qr[j] = *reinterpret_cast<const uint16_t*>(&b);
    }
  }
}

// E4M3 codes and row scales: rows b, b + G, ... per block; the row's
// absolute maximum (the row is read through L2, so that its second reading
// for the codes finds it there), the scale s = fl32(amax / 448), then the
// codes E4M3_satfinite(fl32(A_ij / s)), four per 16-byte load when A and Q
// rows allow it.
__global__ void __launch_bounds__(kThreads)
    quantize_e4m3_kernel(int64_t m, int64_t n, const float* __restrict__ A, int64_t lda,
                         uint8_t* __restrict__ Q, int64_t ldq, float* __restrict__ scales, bool vec) {
  __shared__ float red[kThreads / 32];
  const int64_t nv = vec ? n / 4 * 4 : 0;  // columns read four at a time
  for (int64_t i = blockIdx.x; i < m; i += gridDim.x) {
    const float* Ar = A + i * lda;
    uint8_t* Qr = Q + i * ldq;
    float amax = 0.f;
    // kQuantE4M3U packs of 16 bytes in flight per thread, then one at a time
    constexpr int QU = kQuantE4M3U;
    constexpr int64_t QS = (int64_t)kThreads * 4;  // columns per pack row
    int64_t j = (int64_t)threadIdx.x * 4;
    for (; j + (QU - 1) * QS < nv; j += QU * QS) {
      float4 a[QU];
#pragma unroll
      for (int q = 0; q < QU; ++q) a[q] = __ldcg(reinterpret_cast<const float4*>(Ar + j + q * QS));
#pragma unroll
      for (int q = 0; q < QU; ++q)
        amax = fmaxf(amax, fmaxf(fmaxf(fabsf(a[q].x), fabsf(a[q].y)), fmaxf(fabsf(a[q].z), fabsf(a[q].w))));
    }
    for (; j < nv; j += QS) {
      const float4 a = __ldcg(reinterpret_cast<const float4*>(Ar + j));
      amax = fmaxf(amax, fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(a.w))));
    }
    for (int64_t jj = nv + threadIdx.x; jj < n; jj += kThreads) amax = fmaxf(amax, fabsf(__ldcg(Ar + jj)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = amax;
    __syncthreads();
    amax = 0.f;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) amax = fmaxf(amax, red[w]);
    const float s = __fdiv_rn(amax, 448.0f);
    if (threadIdx.x == 0) scales[i] = s;
    auto code = [&](float v) -> unsigned {
      return s != 0.f ? (unsigned)__nv_cvt_float_to_fp8(__fdiv_rn(v, s), __NV_SATFINITE, __NV_E4M3) : 0u;
    };
    j = (int64_t)threadIdx.x * 4;
    for (; j + (QU - 1) * QS < nv; j += QU * QS) {
      float4 a[QU];
#pragma unroll
      for (int q = 0; q < QU; ++q) a[q] = __ldcs(reinterpret_cast<const float4*>(Ar + j + q * QS));
#pragma unroll
      for (int q = 0; q < QU; ++q)
        *reinterpret_cast<unsigned*>(Qr + j + q * QS) =
            code(a[q].x) | (code(a[q].y) << 8) | (code(a[q].z) << 16) | (code(a[q].w) << 24);
    }
    for (; j < nv; j += QS) {
      const float4 a = __ldcs(reinterpret_cast<const float4*>(Ar + j));
      *reinterpret_cast<unsigned*>(Qr + j) = code(a.x) | (code(a.y) << 8) | (code(a.z) << 16) | (code(a.w) << 24);
    }
    for (int64_t jj = nv + threadIdx.x; jj < n; jj += kThreads) Qr[jj] = (uint8_t)code(__ldcs(Ar + jj));
  }
}

// ------------------------------------------------------------------ GEMV ---

// Four E4M3 codes (one word, element 0 in the low byte) -> FP32, exactly:
// the conversion to a pair of binary16 values is exact (every E4M3 value,
// subnormals included, is a binary16 normal) and so is the widening.
__device__ __forceinline__ void e4m3x4_to_float(unsigned w, float& f0, float& f1, float& f2, float& f3) {
  unsigned lo, hi;
  asm("{\n .reg .b16 a, b;\n mov.b32 {a, b}, %2;\n cvt.rn.f16x2.e4m3x2 %0, a;\n cvt.rn.f16x2.e4m3x2 %1, b;\n}"
      : "=r"(lo), "=r"(hi)
      : "r"(w));
  const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&lo));
  const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&hi));
  f0 = a.x;
  f1 = a.y;
  f2 = b.x;
  f3 = b.y;
}

// Elements 4k .. 4k+3 of a 16-byte pack.
template <int FMT>
__device__ __forceinline__ void unpack4(const uint4& w, int k, float& f0, float& f1, float& f2, float& f3) {
  if constexpr (FMT == 0) {
    const unsigned w0 = k == 0 ? w.x : w.z, w1 = k == 0 ? w.y : w.w;
    f0 = __uint_as_float(w0 << 16);
    f1 = __uint_as_float(w0 & 0xFFFF0000u);
    f2 = __uint_as_float(w1 << 16);
    f3 = __uint_as_float(w1 & 0xFFFF0000u);
  } else {
    e4m3x4_to_float(k == 0 ? w.x : k == 1 ? w.y : k == 2 ? w.z : w.w, f0, f1, f2, f3);
  }
}

// Unit u = (row group u / S of R consecutive rows, chunk u % S of the
// columns); block b takes the units b, b + G, b + 2G, ....  Each load of x serves
// the R rows of the group: with one byte per element, reading x once per row
// would cost four times the matrix's own traffic in L1.  A row's products
// are FP32 fmas in chains of at most 32, folded into a compensated FP32 sum,
// then a fixed-order block sum; a group's missing rows (past m) re-read row
// m-1 and are dropped.
template <int FMT, int R, int U, int MINB, bool OFF32>
__global__ void __launch_bounds__(kThreads, MINB)
    gemv_q_kernel(int64_t m, int64_t n, float alpha, const unsigned char* __restrict__ Q,
                  int64_t ldq_bytes, const float* __restrict__ scales, const float* __restrict__ x,
                  float* __restrict__ c, const Split sp, int64_t KC, int64_t units) {
  constexpr int PER = Fmt<FMT>::PER;
  constexpr int EB = Fmt<FMT>::BYTES;
  constexpr int64_t STEP = (int64_t)kThreads * PER;               // columns per pack position
  constexpr int CHAIN = 32 / (U * PER) > 0 ? 32 / (U * PER) : 1;  // bodies per FP32 chain
  __shared__ float red[R][kThreads / 32];
  __shared__ double red_d[kThreads / 32];
  __shared__ int flag;

  const int S = sp.S;
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {  // interleaved units
    const int64_t g = u / S;
    const int s = (int)(u - g * S);
    const int64_t row0 = g * R;
    const int64_t k0 = (int64_t)s * KC;
    const int64_t k1 = (k0 + KC < n) ? k0 + KC : n;
    const int64_t kv1 = k0 + ((k1 - k0) / PER) * PER;
    // the group's rows: 32-bit offsets from its first row when they fit
    // (fewer registers), else pointers
    const unsigned char* Q0 = Q + row0 * ldq_bytes;
    typename std::conditional<OFF32, unsigned, const unsigned char*>::type rp[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t d = ((row0 + r < m ? row0 + r : m - 1) - row0) * ldq_bytes;
      if constexpr (OFF32) rp[r] = (unsigned)d;
      else rp[r] = Q0 + d;
    }
    auto Qrow = [&](int r) -> const unsigned char* {
      if constexpr (OFF32) return Q0 + rp[r];
      else return rp[r];
    };

    float acc[R], hi[R], lo[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = hi[r] = lo[r] = 0.f;
    int chain = 0;
    int64_t j = k0 + (int64_t)threadIdx.x * PER;
#pragma unroll 1
    for (; j + (U - 1) * STEP < kv1; j += U * STEP) {
      uint4 qp[U][R];
#pragma unroll
      for (int q = 0; q < U; ++q)
#pragma unroll
        for (int r = 0; r < R; ++r)
          qp[q][r] = __ldcs(reinterpret_cast<const uint4*>(Qrow(r) + (j + q * STEP) * EB));
#pragma unroll
      for (int q = 0; q < U; ++q) {
#pragma unroll
        for (int k = 0; k < PER / 4; ++k) {
          const float4 xv = __ldg(reinterpret_cast<const float4*>(x + j + q * STEP + 4 * k));
#pragma unroll
          for (int r = 0; r < R; ++r) {
            float f0, f1, f2, f3;
            unpack4<FMT>(qp[q][r], k, f0, f1, f2, f3);
            acc[r] = __fmaf_rn(f0, xv.x, acc[r]);
            acc[r] = __fmaf_rn(f1, xv.y, acc[r]);
            acc[r] = __fmaf_rn(f2, xv.z, acc[r]);
            acc[r] = __fmaf_rn(f3, xv.w, acc[r]);
          }
        }
      }
      if (++chain == CHAIN) {  // fold each row's chain (at most 32 products) into (hi, lo)
        chain = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          float e;
          two_sum_f(hi[r], acc[r], hi[r], e);
          lo[r] = __fadd_rn(lo[r], e);
          acc[r] = 0.f;
        }
      }
    }
#pragma unroll 1
    for (; j < kv1; j += STEP) {  // remaining whole packs, one at a time
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const uint4 qv = __ldcs(reinterpret_cast<const uint4*>(Qrow(r) + j * EB));
        float a2 = 0.f;
#pragma unroll
        for (int k = 0; k < PER / 4; ++k) {
          const float4 xv = __ldg(reinterpret_cast<const float4*>(x + j + 4 * k));
          float f0, f1, f2, f3;
          unpack4<FMT>(qv, k, f0, f1, f2, f3);
          a2 = __fmaf_rn(f0, xv.x, a2);
          a2 = __fmaf_rn(f1, xv.y, a2);
          a2 = __fmaf_rn(f2, xv.z, a2);
          a2 = __fmaf_rn(f3, xv.w, a2);
        }
        float e;
        two_sum_f(hi[r], a2, hi[r], e);
        lo[r] = __fadd_rn(lo[r], e);
      }
    }
    if (kv1 + threadIdx.x < k1) {  // ragged end (< PER columns)
      const int64_t jj = kv1 + threadIdx.x;
      const float xj = __ldg(x + jj);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float qv = FMT == 0 ? bf16_bits_to_float(reinterpret_cast<const uint16_t*>(Qrow(r))[jj])
                                  : e4m3_bits_to_float(Qrow(r)[jj]);
        acc[r] = __fmaf_rn(qv, xj, acc[r]);
      }
    }

    // fixed-order block sums (warp butterfly, then warps in order) in FP32
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float v = group_sum_f<32>(hi[r] + (lo[r] + acc[r]));
      if ((threadIdx.x & 31) == 0) red[r][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    const int64_t row = row0 + threadIdx.x;  // thread r < R finishes row row0 + r
    const bool mine = threadIdx.x < R && row < m;
    float total = 0.f;
    if (mine) {
#pragma unroll
      for (int w = 0; w < kThreads / 32; ++w) total = __fadd_rn(total, red[threadIdx.x][w]);
    }
    if (S == 1) {
      if (mine) c[row] = __fmaf_rn(alpha, __fmul_rn(FMT == 1 ? scales[row] : 1.f, total), c[row]);
      continue;
    }
    if (mine) sp.part[(int64_t)s * m + row] = (double)total;
    if (arrive_last(sp.tickets + g, (unsigned)S, &flag)) {
      for (int r = 0; r < R && row0 + r < m; ++r) {
        const int64_t rr = row0 + r;
        double p = 0.0;
        for (int q = threadIdx.x; q < S; q += kThreads) p = __dadd_rn(p, __ldcg(sp.part + (int64_t)q * m + rr));
        p = group_sum<32>(p);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red_d[threadIdx.x >> 5] = p;
        __syncthreads();
        if (threadIdx.x == 0) {
          double t = 0.0;
#pragma unroll
          for (int w = 0; w < kThreads / 32; ++w) t = __dadd_rn(t, red_d[w]);
          c[rr] = __fmaf_rn(alpha, __fmul_rn(FMT == 1 ? scales[rr] : 1.f, (float)t), c[rr]);
        }
      }
      if (threadIdx.x == 0) sp.tickets[g] = 0u;
    }
  }
}

}  // namespace

int quantize_bf16_launch(int64_t m, int64_t n, const float* A, int64_t lda, uint16_t* Q,
                         int64_t ldq, cudaStream_t st) {
  const bool vec = (reinterpret_cast<uintptr_t>(A) & 15u) == 0 && (reinterpret_cast<uintptr_t>(Q) & 15u) == 0 &&
                   lda % 4 == 0 && ldq % 8 == 0;
  const int64_t chunks = (n + kQChunk - 1) / kQChunk;
  const int grid = grid_size((const void*)quantize_bf16_kernel, m * chunks);
  quantize_bf16_kernel<<<grid, kThreads, 0, st>>>(m, n, A, lda, Q, ldq, chunks, vec);
  return 0;
}

int quantize_e4m3_launch(int64_t m, int64_t n, const float* A, int64_t lda, uint8_t* Q,
                         int64_t ldq, float* scales, cudaStream_t st) {
  const bool vec = (reinterpret_cast<uintptr_t>(A) & 15u) == 0 && (reinterpret_cast<uintptr_t>(Q) & 3u) == 0 &&
                   lda % 4 == 0 && ldq % 4 == 0;
  const int grid = grid_size((const void*)quantize_e4m3_kernel, m);
  quantize_e4m3_kernel<<<grid, kThreads, 0, st>>>(m, n, A, lda, Q, ldq, scales, vec);
  return 0;
}

int gemv_q_launch(int fmt, int64_t m, int64_t n, float alpha, const void* Q, int64_t ldq,
                  const float* scales, const float* x, float* c, const Split& sp, int64_t kc,
                  int64_t units, cudaStream_t st) {
  const unsigned char* q = static_cast<const unsigned char*>(Q);
  const int64_t ldq_bytes = ldq * (fmt == 0 ? 2 : 1);
  const bool off32 = (kQuantRows[fmt] - 1) * ldq_bytes <= (int64_t)UINT32_MAX;
  auto go = [&](auto kern) {
    const int grid = grid_size((const void*)kern, units);
    kern<<<grid, kThreads, 0, st>>>(m, n, alpha, q, ldq_bytes, scales, x, c, sp, kc, units);
  };
  if (fmt == 0) {
    if (off32) go(gemv_q_kernel<0, kQuantRows[0], kQuantPacks[0], kQuantMinBlocks[0], true>);
    else go(gemv_q_kernel<0, kQuantRows[0], kQuantPacks[0], kQuantMinBlocks[0], false>);
  } else {
    if (off32) go(gemv_q_kernel<1, kQuantRows[1], kQuantPacks[1], kQuantMinBlocks[1], true>);
    else go(gemv_q_kernel<1, kQuantRows[1], kQuantPacks[1], kQuantMinBlocks[1], false>);
  }
  return 0;
}

}  // namespace gb
