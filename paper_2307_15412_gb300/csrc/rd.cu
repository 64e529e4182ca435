// rd.cu -- range-Doppler map of the IF cube.
//
// Two passes of in-place radix-2 decimation-in-time FFTs with the + kernel
// in shared memory, spread over many CTAs:
//   k_rd_rows  R (channel, chirp) rows per CTA: window, FFT over the N
//              samples (range), written to the output cube;
//   k_rd_cols  one CTA per (channel, group of columns): FFT over the M
//              chirps (Doppler) of each column, in place, with the Doppler
//              axis fft-shifted on the way out.
// Twiddles come from sincospi on exact dyadic arguments, once per CTA into
// a shared-memory table (the Hann windows likewise).
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

// x <- u + w v, y <- u - w v with the twiddle w = (cos, sin)
__device__ __forceinline__ void butterfly(float2 *a, float2 *b, float2 w) {
  const float2 u = *a, x = *b;
  const float2 v = make_float2(x.x * w.x - x.y * w.y, x.x * w.y + x.y * w.x);
  *a = make_float2(u.x + v.x, u.y + v.y);
  *b = make_float2(u.x - v.x, u.y - v.y);
}

// tw[k] = e^{+j 2 pi k / L}, k < L / 2 (the twiddle of butterfly pos in a
// stage of length len is tw[pos * L / len]: the same dyadic argument)
__device__ __forceinline__ void twiddles(float2 *tw, int L) {
  for (int k = threadIdx.x; k < (L >> 1); k += blockDim.x) {
    float s, c;
    sincospif(2.f * (float)k / (float)L, &s, &c);
    tw[k] = make_float2(c, s);
  }
}

// R rows of N samples per CTA: window, bit-reversed load, log2 N stages.
// Shared memory: tw[N/2] float2 | rows[R][N] float2 | hann_n[N] | hann_m[R] floats.
__global__ void k_rd_rows(const float2 *__restrict__ in, int rows, int M, int N, int ln, int R, int window,
                          float2 *__restrict__ out) {
  extern __shared__ float2 sm[];
  float2 *tw = sm;
  float2 *row = tw + (N >> 1);
  float *hn = reinterpret_cast<float *>(row + R * N);
  float *hm = hn + N;
  const int r0 = blockIdx.x * R;
  const int nr = min(R, rows - r0);
  twiddles(tw, N);
  if (window == 1) {
    for (int e = threadIdx.x; e < N; e += blockDim.x) hn[e] = hann(e, N);
    for (int r = threadIdx.x; r < nr; r += blockDim.x) hm[r] = hann((r0 + r) % M, M);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nr * N; idx += blockDim.x) {
    const int r = idx >> ln, e = idx & (N - 1);
    float2 v = in[(int64_t)(r0 + r) * N + e];
    if (window == 1) {
      const float w = hm[r] * hn[e];
      v.x *= w;
      v.y *= w;
    }
    row[r * N + bitrev(e, ln)] = v;
  }
  __syncthreads();
  const int hN = N >> 1;
  for (int st = 0; st < ln; ++st) {  // len = 2 << st, half = 1 << st
    for (int b = threadIdx.x; b < nr * hN; b += blockDim.x) {
      const int r = b >> (ln - 1), bb = b & (hN - 1);
      const int grp = bb >> st, pos = bb & ((1 << st) - 1);
      const int i0 = r * N + (grp << (st + 1)) + pos;
      butterfly(&row[i0], &row[i0 + (1 << st)], tw[pos << (ln - 1 - st)]);
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < nr * N; idx += blockDim.x) out[(int64_t)r0 * N + idx] = row[idx];
}

// Doppler: CW columns of one channel per CTA, M chirps each, in place, the
// Doppler axis fft-shifted on the way out.  Shared memory: tw[M/2] | col[M][CW].
__global__ void k_rd_cols(float2 *__restrict__ io, int M, int N, int lm, int CW) {
  extern __shared__ float2 sm[];
  float2 *tw = sm;
  float2 *col = tw + (M >> 1);
  const int groups = (N + CW - 1) / CW;
  const int j = blockIdx.x / groups;
  const int c0 = (blockIdx.x % groups) * CW;
  const int cw = min(CW, N - c0);
  float2 *base = io + (int64_t)j * M * N + c0;
  twiddles(tw, M);
  for (int e = threadIdx.x; e < M * cw; e += blockDim.x) {
    const int m = e / cw, c = e - m * cw;
    col[bitrev(m, lm) * CW + c] = base[(int64_t)m * N + c];
  }
  __syncthreads();
  for (int st = 0; st < lm; ++st) {
    for (int b = threadIdx.x; b < (M >> 1) * cw; b += blockDim.x) {
      const int q = b / cw, c = b - q * cw;
      const int grp = q >> st, pos = q & ((1 << st) - 1);
      const int i0 = (grp << (st + 1)) + pos;
      butterfly(&col[i0 * CW + c], &col[(i0 + (1 << st)) * CW + c], tw[pos << (lm - 1 - st)]);
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
  // rows: R rows of N samples per CTA (about 2048 complex samples)
  const int R = N >= 2048 ? 1 : 2048 / N;
  const int rows = n_rx * M;
  const int rthreads = 256;
  const size_t rsmem = (size_t)(N / 2 + R * N) * sizeof(float2) + (size_t)(N + R) * sizeof(float);
  k_rd_rows<<<(rows + R - 1) / R, rthreads, rsmem, st>>>(reinterpret_cast<const float2 *>(in), rows, M, N, ilog2(N), R,
                                                         window, reinterpret_cast<float2 *>(out));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || M == 1) return e;
  int CW = 4096 / M;  // <= 32 KB of shared memory per CTA
  if (CW > 32) CW = 32;
  if (CW < 1) CW = 1;
  if (CW > N) CW = N;
  const int groups = (N + CW - 1) / CW;
  k_rd_cols<<<n_rx * groups, 256, (size_t)(M / 2 + M * CW) * sizeof(float2), st>>>(reinterpret_cast<float2 *>(out), M,
                                                                                    N, ilog2(M), CW);
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
