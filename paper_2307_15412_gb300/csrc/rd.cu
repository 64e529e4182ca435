// rd.cu -- range-Doppler map of the IF cube.
//
// One CTA per receive channel holds the whole M x N chirp/sample plane in
// shared memory (rows padded by one complex against bank conflicts) and
// runs in-place radix-2 decimation-in-time FFTs with the + kernel: first
// along samples (range), then along chirps (Doppler).  The window is
// applied at load, the Doppler axis is fft-shifted at store.  Twiddles come
// from sincospi on exact dyadic arguments.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rr_internal.cuh"

namespace rr {
namespace {

constexpr int kRdThreads = 1024;

__device__ __forceinline__ int bitrev(int x, int bits) { return bits == 0 ? 0 : (int)(__brev((unsigned)x) >> (32 - bits)); }

__device__ __forceinline__ float hann(int i, int L) {
  if (L <= 1) return 1.f;
  return 0.5f - 0.5f * cospif(2.f * (float)i / (float)(L - 1));
}

__global__ void __launch_bounds__(kRdThreads)
k_range_doppler(const float2 *__restrict__ in, int M, int N, int lm, int ln, int window,
                float2 *__restrict__ out) {
  extern __shared__ float2 sm[];
  const int j = blockIdx.x;
  const int ld = N + 1;
  const float2 *src = in + (int64_t)j * M * N;
  const int tot = M * N;
  // load rows in bit-reversed sample order, windowed
  for (int e = threadIdx.x; e < tot; e += kRdThreads) {
    const int m = e / N, n = e - m * N;
    float2 v = src[e];
    if (window == 1) {
      const float w = hann(n, N) * hann(m, M);
      v.x *= w;
      v.y *= w;
    }
    sm[bitrev(m, lm) * ld + bitrev(n, ln)] = v;  // rows also bit-reversed for the Doppler pass
  }
  __syncthreads();
  // range FFT along n on every row
  for (int len = 2; len <= N; len <<= 1) {
    const int half = len >> 1;
    for (int b = threadIdx.x; b < M * (N >> 1); b += kRdThreads) {
      const int row = b / (N >> 1), q = b - row * (N >> 1);
      const int grp = q / half, pos = q - grp * half;
      const int i0 = row * ld + grp * len + pos, i1 = i0 + half;
      float s, c;
      sincospif(2.f * (float)pos / (float)len, &s, &c);
      const float2 u = sm[i0], x = sm[i1];
      const float2 v = make_float2(x.x * c - x.y * s, x.x * s + x.y * c);
      sm[i0] = make_float2(u.x + v.x, u.y + v.y);
      sm[i1] = make_float2(u.x - v.x, u.y - v.y);
    }
    __syncthreads();
  }
  // Doppler FFT along m on every column
  for (int len = 2; len <= M; len <<= 1) {
    const int half = len >> 1;
    for (int b = threadIdx.x; b < N * (M >> 1); b += kRdThreads) {
      const int col = b % N, q = b / N;
      const int grp = q / half, pos = q - grp * half;
      const int i0 = (grp * len + pos) * ld + col, i1 = i0 + half * ld;
      float s, c;
      sincospif(2.f * (float)pos / (float)len, &s, &c);
      const float2 u = sm[i0], x = sm[i1];
      const float2 v = make_float2(x.x * c - x.y * s, x.x * s + x.y * c);
      sm[i0] = make_float2(u.x + v.x, u.y + v.y);
      sm[i1] = make_float2(u.x - v.x, u.y - v.y);
    }
    __syncthreads();
  }
  float2 *dst = out + (int64_t)j * M * N;
  for (int e = threadIdx.x; e < tot; e += kRdThreads) {
    const int q = e / N, k = e - q * N;
    const int qs = (q + (M >> 1)) & (M - 1);
    dst[qs * N + k] = sm[q * ld + k];
  }
}

int ilog2(int x) {
  int l = 0;
  while ((1 << l) < x) ++l;
  return l;
}

}  // namespace

cudaError_t launch_range_doppler(const float *in, int n_rx, int M, int N, int window, float *out,
                                 cudaStream_t st) {
  const size_t smem = (size_t)M * (N + 1) * sizeof(float2);
  static size_t attr = 0;
  if (smem > 48 * 1024 && smem > attr) {
    cudaError_t e = cudaFuncSetAttribute(k_range_doppler, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = smem;
  }
  k_range_doppler<<<n_rx, kRdThreads, smem, st>>>(reinterpret_cast<const float2 *>(in), M, N, ilog2(M), ilog2(N),
                                                  window, reinterpret_cast<float2 *>(out));
  return cudaGetLastError();
}

}  // namespace rr
