// Device-side twin of synth/__init__.py: the same counter-based SplitMix64
// numbers, written straight into device buffers.  Holds no GEMV/DOT/GER
// arithmetic.  Every launch is a grid-stride loop bounded by n.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

constexpr uint64_t kG = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kM1 = 0xBF58476D1CE4E5B9ull;
constexpr uint64_t kM2 = 0x94D049BB133111EBull;
constexpr uint64_t kS = 0xD1B54A32D192ED03ull;

__host__ __device__ inline uint64_t mix(uint64_t z) {
  z ^= z >> 30; z *= kM1;
  z ^= z >> 27; z *= kM2;
  return z ^ (z >> 31);
}

inline uint64_t key_of(uint64_t seed, uint64_t stream) {
  return mix(mix(seed + kG) ^ (stream * kS));
}

template <typename T>
__device__ inline T to_uniform(uint64_t u);
template <>
__device__ inline double to_uniform<double>(uint64_t u) {
  return (double)(u >> 11) * 0x1p-52 - 1.0;
}
template <>
__device__ inline float to_uniform<float>(uint64_t u) {
  return __fsub_rn(__fmul_rn((float)(uint32_t)(u >> 40), 0x1p-23f), 1.0f);
}

template <typename T>
__global__ void uniform_kernel(T* out, int64_t n, uint64_t key, int64_t offset) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t u = mix(key + (uint64_t)(offset + i + 1) * kG);
    out[i] = to_uniform<T>(u);
  }
}

template <typename T>
__global__ void integers_kernel(T* out, int64_t n, uint64_t key, int64_t offset, int64_t lo,
                                uint64_t span) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t u = mix(key + (uint64_t)(offset + i + 1) * kG) >> 32;
    int64_t r = (int64_t)((u * span) >> 32) + lo;
    out[i] = (T)r;
  }
}

// N(0,1) by Box-Muller (FP32) from the words 2k+1, 2k+2 of the stream, times a
// row scale 10^(lo + (hi - lo) * u_i) with u_i the i-th word of stream + 1.
__global__ void normal_rows_kernel(float* out, int64_t m, int64_t n, uint64_t key, uint64_t rkey,
                                   float lo, float hi) {
  const int64_t total = m * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n;
    const uint64_t w1 = mix(key + (uint64_t)(2 * e + 1) * kG);
    const uint64_t w2 = mix(key + (uint64_t)(2 * e + 2) * kG);
    const float u1 = ((float)(uint32_t)(w1 >> 40) + 1.0f) * 0x1p-24f;  // (0, 1]
    const float u2 = (float)(uint32_t)(w2 >> 40) * 0x1p-24f;           // [0, 1)
    const float z = sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
    const float ur = (float)(uint32_t)(mix(rkey + (uint64_t)(i + 1) * kG) >> 40) * 0x1p-24f;
    out[e] = z * exp10f(lo + (hi - lo) * ur);
  }
}

int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

extern "C" {

int synth_uniform_f64(double* out, int64_t n, uint64_t seed, uint64_t stream, int64_t offset,
                      void* s) {
  if (n <= 0) return 0;
  uniform_kernel<double><<<grid_for(n), 256, 0, (cudaStream_t)s>>>(out, n, key_of(seed, stream), offset);
  return (int)cudaPeekAtLastError();
}

int synth_uniform_f32(float* out, int64_t n, uint64_t seed, uint64_t stream, int64_t offset,
                      void* s) {
  if (n <= 0) return 0;
  uniform_kernel<float><<<grid_for(n), 256, 0, (cudaStream_t)s>>>(out, n, key_of(seed, stream), offset);
  return (int)cudaPeekAtLastError();
}

int synth_integers_f64(double* out, int64_t n, uint64_t seed, uint64_t stream, int64_t offset,
                       int64_t lo, int64_t hi, void* s) {
  if (n <= 0) return 0;
  integers_kernel<double><<<grid_for(n), 256, 0, (cudaStream_t)s>>>(
      out, n, key_of(seed, stream), offset, lo, (uint64_t)(hi - lo + 1));
  return (int)cudaPeekAtLastError();
}

int synth_integers_f32(float* out, int64_t n, uint64_t seed, uint64_t stream, int64_t offset,
                       int64_t lo, int64_t hi, void* s) {
  if (n <= 0) return 0;
  integers_kernel<float><<<grid_for(n), 256, 0, (cudaStream_t)s>>>(
      out, n, key_of(seed, stream), offset, lo, (uint64_t)(hi - lo + 1));
  return (int)cudaPeekAtLastError();
}

int synth_normal_rows_f32(float* out, int64_t m, int64_t n, uint64_t seed, uint64_t stream,
                          float lo, float hi, void* s) {
  if (m <= 0 || n <= 0) return 0;
  normal_rows_kernel<<<grid_for(m * n), 256, 0, (cudaStream_t)s>>>(
      out, m, n, key_of(seed, stream), key_of(seed, stream + 1), lo, hi);
  return (int)cudaPeekAtLastError();
}

}  // extern "C"
