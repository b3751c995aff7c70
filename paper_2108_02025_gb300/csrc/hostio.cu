// Device-to-host copy done by a kernel (include/gbblas.h, gb_copy_to_host).
// Not an operation of the paper: the IO around its GEMV, DOT and GER when the
// caller's operands live in host memory.  The kernel stores straight into
// page-locked host memory through its device mapping, so the copy takes no
// copy engine: it runs beside copy-engine transfers in the other direction
// even where the driver would put both directions on one engine.
#include <cstdint>

#include <cuda_runtime.h>

#include "gbblas.h"

namespace gb {
namespace {

constexpr int kCopyThreads = 512;
constexpr int kCopyUnroll = 4;

// 16-byte words: kCopyUnroll loads in flight per thread, then the rest one
// by one.
__global__ void __launch_bounds__(kCopyThreads) copy16_kernel(const int4* __restrict__ src, int4* __restrict__ dst,
                                                              int64_t words) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + (kCopyUnroll - 1) * stride < words; i += kCopyUnroll * stride) {
    int4 v[kCopyUnroll];
#pragma unroll
    for (int q = 0; q < kCopyUnroll; ++q) v[q] = __ldcs(src + i + q * stride);
#pragma unroll
    for (int q = 0; q < kCopyUnroll; ++q) dst[i + q * stride] = v[q];
  }
  for (; i < words; i += stride) dst[i] = __ldcs(src + i);
}

__global__ void __launch_bounds__(kCopyThreads) copy1_kernel(const unsigned char* __restrict__ src,
                                                             unsigned char* __restrict__ dst, int64_t bytes) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < bytes; i += stride) dst[i] = src[i];
}

int sm_count() {
  static int count = [] {
    int dev = 0, c = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return c;
  }();
  return count;
}

}  // namespace
}  // namespace gb

using namespace gb;

extern "C" int gb_copy_to_host(void* dst, const void* src, size_t bytes, gb_stream stream) {
  if (bytes == 0) return GB_OK;
  if (!dst) return -1;
  if (!src) return -2;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, dst) != cudaSuccess || at.type != cudaMemoryTypeHost || !at.devicePointer) {
    cudaGetLastError();
    return -1;
  }
  const uintptr_t d = (uintptr_t)at.devicePointer, s = (uintptr_t)src;
  if ((d < s && s - d < bytes) || (s <= d && d - s < bytes)) return -2;
  const int sms = sm_count();
  if (sms <= 0) return GB_ERR_CUDA;
  cudaStream_t sm = static_cast<cudaStream_t>(stream);
  unsigned char* dd = static_cast<unsigned char*>(at.devicePointer);
  const unsigned char* ss = static_cast<const unsigned char*>(src);
  if (d % 16 == 0 && s % 16 == 0) {
    const int64_t words = (int64_t)(bytes / 16);
    if (words > 0) {
      const int64_t want = (words + kCopyThreads - 1) / kCopyThreads;
      const unsigned grid = (unsigned)(want < 2 * sms ? want : 2 * sms);
      copy16_kernel<<<grid, kCopyThreads, 0, sm>>>(reinterpret_cast<const int4*>(ss), reinterpret_cast<int4*>(dd),
                                                   words);
    }
    const int64_t rest = (int64_t)(bytes % 16);
    if (rest > 0) copy1_kernel<<<1, 32, 0, sm>>>(ss + 16 * words, dd + 16 * words, rest);
  } else {
    const int64_t want = ((int64_t)bytes + kCopyThreads - 1) / kCopyThreads;
    const unsigned grid = (unsigned)(want < 2 * sms ? want : 2 * sms);
    copy1_kernel<<<grid, kCopyThreads, 0, sm>>>(ss, dd, (int64_t)bytes);
  }
  return cudaPeekAtLastError() == cudaSuccess ? GB_OK : GB_ERR_CUDA;
}
