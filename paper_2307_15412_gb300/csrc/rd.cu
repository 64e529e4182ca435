// rd.cu -- range-Doppler map of the IF cube.
//
// Two passes of in-place radix-2 decimation-in-time FFTs with the + kernel
// in shared memory, spread over many CTAs:
//   k_rd_rows  one CTA per (channel, chirp) row: window, FFT over the N
//              samples (range), written to the output cube;
//   k_rd_cols  one CTA per (channel, group of columns): FFT over the M
//              chirps (Doppler) of each column, in place, with the Doppler
//              axis fft-shifted on the way out.
// Twiddles come from sincospi on exact dyadic arguments.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rr_internal.cuh"

namespace rr {
namespace {

__device__ __forceinline__ int bitrev(int x, int bits) { return bits == 0 ? 0 : (int)(__brev((unsigned)x) >> (32 - bits)); }

__device__ __forceinline__ float hann(int i, int L) {
  if (L <= 1) return 1.f;
  return 0.5f - 0.5f * cospif(2.f * (float)i / (float)(L - 1));
}

__device__ __forceinline__ void butterfly(float2 *a, float2 *b, int pos, int len) {
  float s, c;
  sincospif(2.f * (float)pos / (float)len, &s, &c);
  const float2 u = *a, x = *b;
  const float2 v = make_float2(x.x * c - x.y * s, x.x * s + x.y * c);
  *a = make_float2(u.x + v.x, u.y + v.y);
  *b = make_float2(u.x - v.x, u.y - v.y);
}

__global__ void k_rd_rows(const float2 *__restrict__ in, int M, int N, int ln, int window, float2 *__restrict__ out) {
  extern __shared__ float2 row[];
  const int rix = blockIdx.x;  // j * M + m
  const int m = rix % M;
  const float wm = window == 1 ? hann(m, M) : 1.f;
  const float2 *src = in + (int64_t)rix * N;
  for (int e = threadIdx.x; e < N; e += blockDim.x) {
    float2 v = src[e];
    if (window == 1) {
      const float w = wm * hann(e, N);
      v.x *= w;
      v.y *= w;
    }
    row[bitrev(e, ln)] = v;
  }
  __syncthreads();
  for (int len = 2; len <= N; len <<= 1) {
    const int half = len >> 1;
    for (int b = threadIdx.x; b < (N >> 1); b += blockDim.x) {
      const int grp = b / half, pos = b - grp * half;
      const int i0 = grp * len + pos;
      butterfly(&row[i0], &row[i0 + half], pos, len);
    }
    __syncthreads();
  }
  float2 *dst = out + (int64_t)rix * N;
  for (int e = threadIdx.x; e < N; e += blockDim.x) dst[e] = row[e];
}

__global__ void k_rd_cols(float2 *__restrict__ io, int M, int N, int lm, int CW) {
  extern __shared__ float2 col[];  // [M][CW]
  const int groups = (N + CW - 1) / CW;
  const int j = blockIdx.x / groups;
  const int c0 = (blockIdx.x % groups) * CW;
  const int cw = min(CW, N - c0);
  float2 *base = io + (int64_t)j * M * N + c0;
  for (int e = threadIdx.x; e < M * cw; e += blockDim.x) {
    const int m = e / cw, c = e - m * cw;
    col[bitrev(m, lm) * CW + c] = base[(int64_t)m * N + c];
  }
  __syncthreads();
  for (int len = 2; len <= M; len <<= 1) {
    const int half = len >> 1;
    for (int b = threadIdx.x; b < (M >> 1) * cw; b += blockDim.x) {
      const int q = b / cw, c = b - q * cw;
      const int grp = q / half, pos = q - grp * half;
      const int i0 = grp * len + pos;
      butterfly(&col[i0 * CW + c], &col[(i0 + half) * CW + c], pos, len);
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < M * cw; e += blockDim.x) {
    const int q = e / cw, c = e - q * cw;
    const int qs = (q + (M >> 1)) & (M - 1);
    base[(int64_t)qs * N + c] = col[q * CW + c];
  }
}

// out[f][j][c] = in[f][j][c] conj(in[f][0][c]) / |in[f][0][c]| (c = cell)
__global__ void k_phase_reference(const float2 *__restrict__ in, int64_t n_frames, int n_rx, int64_t cells,
                                  float2 *__restrict__ out) {
  const int64_t total = n_frames * cells;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = i / cells, c = i - f * cells;
    const float2 r = in[f * n_rx * cells + c];
    const float mag = hypotf(r.x, r.y);
    const float ux = mag > 0.f ? r.x / mag : 1.f, uy = mag > 0.f ? -r.y / mag : 0.f;  // conj(r) / |r|
    for (int j = 0; j < n_rx; ++j) {
      const int64_t o = (f * n_rx + j) * cells + c;
      const float2 v = in[o];
      out[o] = make_float2(v.x * ux - v.y * uy, v.x * uy + v.y * ux);
    }
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
  const int rthreads = N / 2 < 32 ? 32 : (N / 2 > 512 ? 512 : N / 2);
  k_rd_rows<<<n_rx * M, rthreads, N * sizeof(float2), st>>>(reinterpret_cast<const float2 *>(in), M, N, ilog2(N),
                                                            window, reinterpret_cast<float2 *>(out));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || M == 1) return e;
  int CW = 4096 / M;  // <= 32 KB of shared memory per CTA
  if (CW > 32) CW = 32;
  if (CW < 1) CW = 1;
  if (CW > N) CW = N;
  const int groups = (N + CW - 1) / CW;
  k_rd_cols<<<n_rx * groups, 256, (size_t)M * CW * sizeof(float2), st>>>(reinterpret_cast<float2 *>(out), M, N,
                                                                         ilog2(M), CW);
  return cudaGetLastError();
}

cudaError_t launch_phase_reference(const float *in, int64_t n_frames, int n_rx, int64_t cells, float *out,
                                   cudaStream_t st) {
  int sms = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (n_frames * cells + 255) / 256;
  const int blocks = (int)(want < 1 ? 1 : (want > 8 * sms ? 8 * sms : want));
  k_phase_reference<<<blocks, 256, 0, st>>>(reinterpret_cast<const float2 *>(in), n_frames, n_rx, cells,
                                            reinterpret_cast<float2 *>(out));
  return cudaGetLastError();
}

}  // namespace rr
